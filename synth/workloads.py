"""Named synthetic workloads: matrix recipe, interval and subspace size.

Seeds are 20260401 + workload index.  The matrices and draws come from
``synth.matrices`` and ``synth.rng``; nothing here computes eigenvalues.
Intervals that need the spectrum of the matrix (the 2D case) are read from
``tests/golden``, written there by a script that calls the oracle only.
"""
from __future__ import annotations

import json
import os
from dataclasses import dataclass

import numpy as np

from . import matrices

BASE_SEED = 20260401
_GOLDEN = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                       "tests", "golden")


@dataclass
class Workload:
    name: str
    seed: int
    p: int
    a: float
    b: float
    is_complex: bool
    description: str

    def matrix(self) -> matrices.CSR:
        return _BUILDERS[self.name](self.seed)


def _c1_matrix(seed):
    return matrices.laplacian2d_dirichlet(32, seed, 0.5)


def _c2_matrix(seed):
    return matrices.anderson(64, 3, 4.0, seed, complex_phases=True)


def _c3_matrix(seed):
    return matrices.ks_like_3d(96, seed, n_wells=64, sigma=1.5)


def _c4_matrix(seed):
    return matrices.anderson(80, 3, 6.0, seed, complex_phases=False)


_BUILDERS = {
    "lap2d_32": _c1_matrix,
    "anderson3d_c_64": _c2_matrix,
    "ks8_96": _c3_matrix,
    "anderson3d_r_80": _c4_matrix,
}


def _golden_interval(name):
    path = os.path.join(_GOLDEN, f"interval_{name}.json")
    with open(path) as f:
        d = json.load(f)
    return float(d["a"]), float(d["b"])


def lap2d_32() -> Workload:
    """2D 5-point Dirichlet Laplacian, 32 x 32 (n = 1024), potential U[-0.5, 0.5];
    interval around the spectrum midpoint holding about 16 eigenvalues; p = 24."""
    a, b = _golden_interval("lap2d_32")
    return Workload("lap2d_32", BASE_SEED + 0, 24, a, b, False,
                    "2D Laplacian 32^2 Dirichlet + U[-0.5,0.5], real FP64, p=24")


# Half-width of the interval around E = 0 for the 64^3 complex Anderson model:
# a kernel-polynomial estimate of the density of states at E = 0 (3000 Jackson
# moments, 6 random-phase vectors) puts about 99 eigenvalues in [-0.0017, 0.0017].
ANDERSON64_HALFWIDTH = 0.0017


def anderson3d_c_64() -> Workload:
    """Complex Hermitian 3D Anderson model, 64^3 periodic (n = 262,144), random
    U(1) Peierls phases, on-site disorder U[-2, 2]; interval [-0.0017, 0.0017]
    (about 100 eigenvalues); p = 160."""
    h = ANDERSON64_HALFWIDTH
    return Workload("anderson3d_c_64", BASE_SEED + 1, 160, -h, h, True,
                    "3D Anderson 64^3 periodic, Peierls phases, W=4, complex, p=160")


def anderson3d_c_48() -> Workload:
    """The 64^3 workload's model on a 48^3 grid (n = 110,592), p = 160: a
    smaller case for kernel profiling whose blocks (141 MB in FP32 complex)
    still exceed L2."""
    h = ANDERSON64_HALFWIDTH
    return Workload("anderson3d_c_48", BASE_SEED + 11, 160, -h, h, True,
                    "3D Anderson 48^3 periodic, Peierls phases, W=4, complex, p=160")


_BUILDERS["anderson3d_c_48"] = lambda seed: matrices.anderson(48, 3, 4.0, seed, complex_phases=True)


def anderson3d_c_40() -> Workload:
    """The 64^3 workload's model on a 40^3 grid (n = 64,000), p = 160, with the
    interval widened by the ratio of the sizes (262,144 / 64,000) so that it
    holds about the same number of eigenvalues (about 100) at the same density
    of states: the case on which the plain FP64 path and the FP32 forms are
    timed against each other (its FP32 blocks, 82 MB, and the three of them
    that one step touches still exceed what L2 keeps)."""
    h = ANDERSON64_HALFWIDTH * 262144.0 / 64000.0
    return Workload("anderson3d_c_40", BASE_SEED + 13, 160, -h, h, True,
                    "3D Anderson 40^3 periodic, Peierls phases, W=4, complex, p=160")


_BUILDERS["anderson3d_c_40"] = lambda seed: matrices.anderson(40, 3, 4.0, seed, complex_phases=True)

def ks8_96() -> Workload:
    """Real symmetric Kohn-Sham-like Hamiltonian on a 96^3 periodic grid
    (n = 884,736): -1/2 times the eighth-order Laplacian (25 nonzeros per row)
    plus 64 negative Gaussian wells (sigma = 1.5 grid units, seeded centres).
    Interval [E_300, E_500] from the oracle's count estimate (stored in
    tests/golden): about 200 eigenvalues around the midpoint of the
    300th-500th; p = 300."""
    a, b = _golden_interval("ks8_96")
    return Workload("ks8_96", BASE_SEED + 2, 300, a, b, False,
                    "Kohn-Sham-like 96^3 periodic, 8th-order stencil + 64 Gaussian wells, real, p=300")


@dataclass
class SliceWorkload:
    """Several disjoint intervals of one matrix (spectrum slicing)."""
    name: str
    seed: int
    a: list
    b: list
    p: list          # 0 = estimated (Sec. 3.4)
    is_complex: bool
    description: str

    def matrix(self) -> matrices.CSR:
        return _BUILDERS[self.name](self.seed)


def anderson3d_r_48_slices() -> SliceWorkload:
    """Real 3D Anderson model, 48^3 periodic (n = 110,592), on-site disorder
    U[-3, 3]; eight contiguous slices of equal width around E = 0 holding about
    30 eigenvalues each (window from the oracle's count estimate, stored in
    tests/golden); subspace sizes estimated (p = 0)."""
    path = os.path.join(_GOLDEN, "slices_anderson3d_r_48.json")
    with open(path) as f:
        d = json.load(f)
    n = len(d["a"])
    # neighbouring slices share an end: move each slice's upper end one ulp down
    # so that the slices are disjoint
    b = [float(np.nextafter(x, -np.inf)) for x in d["b"]]
    return SliceWorkload("anderson3d_r_48_slices", BASE_SEED + 12, list(d["a"]), b, [0] * n, False,
                         "3D Anderson 48^3 periodic, W=6, real, 8 slices around E=0, p estimated")


_BUILDERS["anderson3d_r_48_slices"] = lambda seed: matrices.anderson(48, 3, 6.0, seed, complex_phases=False)


def anderson3d_r_80_slices() -> SliceWorkload:
    """Batched spectrum slicing of one real 3D Anderson model, 80^3 periodic
    (n = 512,000), on-site disorder U[-3, 3]: sixteen contiguous slices with
    seeded uneven target counts in [20, 150] (56..141 here, 1,480 in all),
    starting above the 200th eigenvalue, edges from the oracle's count
    estimate (stored in tests/golden); block m = ceil(1.5 count) per slice
    (2,224 columns in all)."""
    import math
    path = os.path.join(_GOLDEN, "slices_anderson3d_r_80.json")
    with open(path) as f:
        d = json.load(f)
    b = [float(np.nextafter(x, -np.inf)) for x in d["b"]]
    p = [int(math.ceil(1.5 * c)) for c in d["target_counts"]]
    return SliceWorkload("anderson3d_r_80_slices", BASE_SEED + 3, list(d["a"]), b, p, False,
                         "3D Anderson 80^3 periodic, W=6, real, 16 slices above the 200th eigenvalue, "
                         "p = 1.5 count")


_BUILDERS["anderson3d_r_80_slices"] = _c4_matrix

WORKLOADS = {
    "lap2d_32": lap2d_32,
    "anderson3d_c_64": anderson3d_c_64,
    "anderson3d_c_48": anderson3d_c_48,
    "anderson3d_c_40": anderson3d_c_40,
    "ks8_96": ks8_96,
}

SLICE_WORKLOADS = {
    "anderson3d_r_48_slices": anderson3d_r_48_slices,
    "anderson3d_r_80_slices": anderson3d_r_80_slices,
}


@dataclass
class Request:
    """One serving request: a matrix recipe, an interval, p = 0 (estimated)."""
    dim: int
    L: int
    W: float
    is_complex: bool
    seed: int
    a: float
    b: float
    target: int

    def matrix(self) -> matrices.CSR:
        return matrices.anderson(self.L, self.dim, self.W, self.seed, complex_phases=self.is_complex)


def serving_requests(count: int = 24, seed: int = BASE_SEED + 5, n_lo: float = 1e4,
                     n_hi: float = 1e5, count_hi: int = 64) -> list:
    """A seeded stream of independent eigenproblems: Anderson models in 2D or
    3D (50/50), real or complex (50/50), n log-uniform in [n_lo, n_hi]
    (L = round(n^(1/d))), disorder W ~ U[1, 6], a target count U{8..count_hi} and an
    interval of that many states under a flat density of states over the
    Gershgorin range [-2d - W/2, 2d + W/2], centred uniformly in the middle
    half of the band.  The true count differs from the target where the
    density is not flat; the requests leave p = 0 (estimated)."""
    import math
    import numpy as np
    from . import rng
    u = rng.uniform(seed, rng.STREAM_TEST, np.arange(7 * count, dtype=np.uint64)).reshape(count, 7)
    out = []
    for i in range(count):
        dim = 2 if u[i, 0] < 0.5 else 3
        is_c = bool(u[i, 1] < 0.5)
        n = math.exp(math.log(n_lo) + u[i, 2] * (math.log(n_hi) - math.log(n_lo)))
        L = max(3, int(round(n ** (1.0 / dim))))
        W = 1.0 + 5.0 * u[i, 3]
        target = 8 + int((count_hi - 7) * u[i, 4])
        span = 4.0 * dim + W
        half = 0.5 * target * span / (L ** dim)
        centre = (u[i, 5] - 0.5) * 0.5 * span
        out.append(Request(dim, L, W, is_c, seed + 1 + i, centre - half, centre + half, target))
    return out
