"""Eigenvalue count estimate and subspace size (Sec. 3.4).

TEST INFRASTRUCTURE (see ``oracle/__init__``).  The count e~ of eigenvalues
in [a, b] is the trace of an approximate spectral projector, here the filter
rho_k(l(A)) of Alg. 2 at the maximum degree k, estimated stochastically:
tr(M) ~ (1/m) sum_c z_c^H M z_c over m probe vectors with E[z z^H] = I
(Hutchinson, Commun. Stat. Simul. Comput. 18, 1989).  The subspace size is
then p = ceil(mu e~).

Readings taken where the paper is silent:

* the probes are real Rademacher vectors (entries +-1, equally likely), passed
  in as an n x m block Z; the number m is a parameter (32 by default on the
  GPU side);
* a non-positive or tiny estimate still gives a usable size: p = ceil(mu
  max(e~, 1)), clipped to [1, min(n, p_max)].
"""
from __future__ import annotations

import math

import numpy as np

from .filter import clenshaw_apply


def trace_estimate(A, coef: np.ndarray, l1: float, l2: float, Z: np.ndarray) -> float:
    """(1/m) sum_c Re(z_c^H rho(l(A)) z_c) with rho(x) = sum_j a_j T_j(x) (Alg. 2)."""
    m = Z.shape[1]
    Y = clenshaw_apply(A, coef, l1, l2, Z)
    return float(np.sum(np.real(np.conj(Z) * Y)) / m)


def subspace_size(e_est: float, mu: float, n: int, p_max: int) -> int:
    """p = ceil(mu e~) (Sec. 3.4), with e~ floored at 1 and p clipped to [1, min(n, p_max)]."""
    p = int(math.ceil(mu * max(e_est, 1.0)))
    return max(1, min(p, n, p_max))


def chebyshev_trace_moments(A, l1: float, l2: float, Z: np.ndarray, k: int) -> np.ndarray:
    """mu_j = (1/m) sum_c Re(z_c^H T_j(l(A)) z_c), j = 0..k, by the three-term
    recurrence T_{j+1}(x) = 2 x T_j(x) - T_{j-1}(x) on the probe block.

    Since rho = sum_j a_j T_j is linear in the T_j, sum_j a_j mu_j equals
    ``trace_estimate(A, a, l1, l2, Z)`` for the same probes: one pass gives the
    Hutchinson estimate of every filter of degree <= k (the kernel polynomial
    method's moments, Weisse et al., Rev. Mod. Phys. 78, 2006)."""
    m = Z.shape[1]
    mu = np.zeros(k + 1)
    T0 = np.array(Z, dtype=np.float64 if not np.iscomplexobj(Z) else np.complex128, copy=True)
    mu[0] = float(np.sum(np.real(np.conj(Z) * T0)) / m)
    if k == 0:
        return mu
    T1 = l1 * (A @ T0) + l2 * T0
    mu[1] = float(np.sum(np.real(np.conj(Z) * T1)) / m)
    for j in range(2, k + 1):
        T0, T1 = T1, 2.0 * (l1 * (A @ T1) + l2 * T1) - T0
        mu[j] = float(np.sum(np.real(np.conj(Z) * T1)) / m)
    return mu
