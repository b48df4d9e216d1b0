"""Write the stored expected values under tests/golden from the oracle only.

Run from the repository root:  python tests/golden/make_golden.py

* interval_lap2d_32.json -- the interval of the 32 x 32 2D Laplacian workload,
  chosen from the dense spectrum (oracle.dense): endpoints at the midpoints of
  the gaps around a run of 14-18 eigenvalues near the spectrum midpoint,
  taking the run whose two bounding gaps are widest; plus the eigenvalues
  inside it.
"""
from __future__ import annotations

import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import dense  # noqa: E402
from synth import matrices  # noqa: E402
from synth.workloads import BASE_SEED  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))


def lap2d_interval():
    A = matrices.laplacian2d_dirichlet(32, BASE_SEED + 0, 0.5)
    lam = dense.all_eigenvalues(A.to_dense())
    n = lam.size
    mid = n // 2
    best = None
    for cnt in range(14, 19):
        for lo in range(mid - cnt // 2 - 3, mid - cnt // 2 + 4):
            hi = lo + cnt
            g = min(lam[lo] - lam[lo - 1], lam[hi] - lam[hi - 1])
            if best is None or g > best[0]:
                best = (g, lo, hi)
    _, lo, hi = best
    a = 0.5 * (lam[lo - 1] + lam[lo])
    b = 0.5 * (lam[hi - 1] + lam[hi])
    out = dict(a=a, b=b, count=int(hi - lo), eigenvalues=[float(x) for x in lam[lo:hi]],
               min_gap=float(best[0]), lambda_min=float(lam[0]), lambda_max=float(lam[-1]),
               source="oracle.dense.all_eigenvalues of synth.matrices.laplacian2d_dirichlet(32, 20260401, 0.5)")
    with open(os.path.join(HERE, "interval_lap2d_32.json"), "w") as f:
        json.dump(out, f, indent=1)
    print("lap2d_32:", a, b, hi - lo, "min gap", best[0])


if __name__ == "__main__":
    lap2d_interval()
