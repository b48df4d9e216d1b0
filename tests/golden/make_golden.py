"""Write the stored expected values under tests/golden from the oracle only.

Run from the repository root:  python tests/golden/make_golden.py

* interval_lap2d_32.json -- the interval of the 32 x 32 2D Laplacian workload,
  chosen from the dense spectrum (oracle.dense): endpoints at the midpoints of
  the gaps around a run of 14-18 eigenvalues near the spectrum midpoint,
  taking the run whose two bounding gaps are widest; plus the eigenvalues
  inside it.
* slices_anderson3d_r_48.json -- eight contiguous spectrum slices around
  E = 0 of the real 48^3 Anderson model (W = 6): the half-width w of the
  window [-w, w] holding about 240 eigenvalues, from the oracle's count
  estimate (oracle.trace: Hutchinson trace of a degree-4000 step filter over
  16 +-1 probes, bounds from the Gershgorin interval), cut into eight slices
  of equal width; and the estimated count of each slice.
* interval_ks8_96.json -- the interval of the 96^3 Kohn-Sham-like workload:
  [E_300, E_500], where E_N is the energy below which the oracle's count
  estimate finds N eigenvalues (oracle.trace: Chebyshev moments of degree
  3000 over 16 +-1 probes, i.e. the Hutchinson trace of the degree-3000 step
  filter of [lambda_min, E], bounds from the Gershgorin interval), so that the
  interval holds about 200 eigenvalues around the midpoint of the 300th-500th.

* slices_anderson3d_r_80.json -- sixteen contiguous slices of the real 80^3
  Anderson model (W = 6) above its 200th eigenvalue with seeded uneven target
  counts in [20, 150], edges from the oracle's count estimate (Chebyshev
  moments of degree 3000 over 16 +-1 probes).

    python tests/golden/make_golden.py [lap2d | slices48 | ks96 | slices80]   (default: all)
"""
from __future__ import annotations

import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import chebyshev as cb  # noqa: E402
from oracle import dense, fsi, trace  # noqa: E402
from synth import matrices, rng  # noqa: E402
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


def _count(A, lo, hi, l1, l2, Z, k):
    coef = cb.filter_coefficients(l1 * lo + l2, l1 * hi + l2, k, cb.DAMP_LANCZOS_M, 0.5)
    return trace.trace_estimate(A, coef, l1, l2, Z)


def slices_anderson48(target=240, nslices=8, k=4000, probes=16):
    seed = BASE_SEED + 12
    A = matrices.anderson(48, 3, 6.0, seed, complex_phases=False).to_scipy()
    lmin, lmax = fsi.gershgorin(A)
    l1, l2 = cb.linear_map(lmin, lmax)
    Z = rng.rademacher_block(seed, rng.STREAM_TEST, A.shape[0], probes)
    # density at E = 0 from a window, then the half-width for `target` states
    w0 = 0.01
    c0 = _count(A, -w0, w0, l1, l2, Z, k)
    w = w0 * target / max(c0, 1.0)
    edges = np.linspace(-w, w, nslices + 1)
    counts = [_count(A, edges[i], edges[i + 1], l1, l2, Z, k) for i in range(nslices)]
    out = dict(a=[float(x) for x in edges[:-1]], b=[float(x) for x in edges[1:]], half_width=float(w),
               count_estimates=[float(c) for c in counts], window_estimate_at_0_01=float(c0),
               source=("oracle.trace.trace_estimate (degree %d, %d probes of stream %d) on "
                       "synth.matrices.anderson(48, 3, 6.0, %d, False); Gershgorin bounds" %
                       (k, probes, rng.STREAM_TEST, seed)))
    with open(os.path.join(HERE, "slices_anderson3d_r_48.json"), "w") as f:
        json.dump(out, f, indent=1)
    print("anderson3d_r_48 slices: w", w, "counts", [round(c, 1) for c in counts])


def ks8_96_interval(lo_count=300, hi_count=500, k=3000, probes=16):
    seed = BASE_SEED + 2
    A = matrices.ks_like_3d(96, seed, n_wells=64, sigma=1.5).to_scipy()
    lmin, lmax = fsi.gershgorin(A)
    l1, l2 = cb.linear_map(lmin, lmax)
    Z = rng.rademacher_block(seed, rng.STREAM_TEST, A.shape[0], probes)
    mu = trace.chebyshev_trace_moments(A, l1, l2, Z, k)

    def below(E):  # estimated number of eigenvalues in [lmin, E]
        coef = cb.filter_coefficients(-1.0, l1 * E + l2, k, cb.DAMP_LANCZOS_M, 0.5)
        return float(coef @ mu)

    def energy_at(count):  # bisection on the monotone estimate
        lo, hi = lmin, lmax
        for _ in range(100):
            mid = 0.5 * (lo + hi)
            if below(mid) < count:
                lo = mid
            else:
                hi = mid
        return 0.5 * (lo + hi)

    a, b = energy_at(lo_count), energy_at(hi_count)
    out = dict(a=a, b=b, count_estimate=below(b) - below(a), lo_count=lo_count, hi_count=hi_count,
               gershgorin=[lmin, lmax], degree=k, probes=probes,
               count_below_zero=below(0.0),
               source=("oracle.trace.chebyshev_trace_moments (degree %d, %d probes of stream %d) on "
                       "synth.matrices.ks_like_3d(96, %d, n_wells=64, sigma=1.5); Gershgorin bounds" %
                       (k, probes, rng.STREAM_TEST, seed)))
    with open(os.path.join(HERE, "interval_ks8_96.json"), "w") as f:
        json.dump(out, f, indent=1)
    print("ks8_96:", a, b, "estimated count", out["count_estimate"])


def slices_anderson80(nslices=16, start_count=200, k=3000, probes=16):
    """Sixteen contiguous slices of the real 80^3 Anderson model (W = 6)
    starting above its 200th eigenvalue (the low end of the band, where the
    density of states is small), with seeded uneven target counts in
    [20, 150]: slice s = [E_{N_s}, E_{N_{s+1}}] with N_0 = 200 and
    N_{s+1} = N_s + count_s, E_N from the oracle's count estimate."""
    seed = BASE_SEED + 3
    A = matrices.anderson(80, 3, 6.0, seed, complex_phases=False).to_scipy()
    lmin, lmax = fsi.gershgorin(A)
    l1, l2 = cb.linear_map(lmin, lmax)
    Z = rng.rademacher_block(seed, rng.STREAM_TEST, A.shape[0], probes)
    mu = trace.chebyshev_trace_moments(A, l1, l2, Z, k)

    def below(E):
        coef = cb.filter_coefficients(-1.0, l1 * E + l2, k, cb.DAMP_LANCZOS_M, 0.5)
        return float(coef @ mu)

    def energy_at(count):
        lo, hi = lmin, lmax
        for _ in range(100):
            mid = 0.5 * (lo + hi)
            if below(mid) < count:
                lo = mid
            else:
                hi = mid
        return 0.5 * (lo + hi)

    u = rng.uniform(seed, rng.STREAM_TEST, np.arange(nslices, dtype=np.uint64))
    counts = [20 + int(131 * x) for x in u]
    cum = [start_count]
    for c in counts:
        cum.append(cum[-1] + c)
    edges = [energy_at(c) for c in cum]
    est = [below(edges[i + 1]) - below(edges[i]) for i in range(nslices)]
    out = dict(a=edges[:-1], b=edges[1:], target_counts=counts, count_estimates=est, start_count=start_count,
               gershgorin=[lmin, lmax], degree=k, probes=probes,
               source=("oracle.trace.chebyshev_trace_moments (degree %d, %d probes of stream %d) on "
                       "synth.matrices.anderson(80, 3, 6.0, %d, False); Gershgorin bounds; counts from "
                       "synth.rng.uniform(%d, stream %d)" % (k, probes, rng.STREAM_TEST, seed, seed,
                                                             rng.STREAM_TEST)))
    with open(os.path.join(HERE, "slices_anderson3d_r_80.json"), "w") as f:
        json.dump(out, f, indent=1)
    print("anderson3d_r_80 slices: edges", [round(e, 4) for e in edges], "counts", counts,
          "estimates", [round(c, 1) for c in est])


if __name__ == "__main__":
    which = sys.argv[1:] or ["lap2d", "slices48", "ks96", "slices80"]
    if "lap2d" in which:
        lap2d_interval()
    if "slices48" in which:
        slices_anderson48()
    if "ks96" in which:
        ks8_96_interval()
    if "slices80" in which:
        slices_anderson80()
