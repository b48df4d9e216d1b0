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

WORKLOADS = {
    "lap2d_32": lap2d_32,
    "anderson3d_c_64": anderson3d_c_64,
    "anderson3d_c_48": anderson3d_c_48,
}
