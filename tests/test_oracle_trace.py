"""Pins of the eigenvalue-count estimate (Sec. 3.4) in oracle/trace.py.

The estimate is a Hutchinson trace of the filter rho_k(l(A)).  It is pinned
by: identity probes (the exact trace, with rho evaluated by its defining
cosine sum on the dense spectrum, not by Clenshaw); the full set of sign
vectors of a tiny matrix (exactly unbiased); random probes within six
standard deviations of the exact trace (variance from the dense filter
matrix); and the count itself for a sharp filter with ends in spectral gaps.
"""
import itertools
import math

import numpy as np
import pytest

from oracle import chebyshev as cb
from oracle import trace
from synth import matrices, rng


def _rho_direct(coef, x):
    j = np.arange(len(coef))
    return np.cos(np.outer(np.arccos(np.clip(x, -1, 1)), j)) @ coef


def _setup(A, a, b, k):
    lam, U = np.linalg.eigh(A.to_dense())
    lmin, lmax = lam[0] - 0.1, lam[-1] + 0.1
    l1, l2 = cb.linear_map(lmin, lmax)
    coef = cb.filter_coefficients(l1 * a + l2, l1 * b + l2, k, cb.DAMP_LANCZOS_M, 0.5)
    return lam, U, l1, l2, coef


def _gap_interval(lam, i, c):
    return 0.5 * (lam[i - 1] + lam[i]), 0.5 * (lam[i + c - 1] + lam[i + c])


@pytest.mark.parametrize("is_complex", [False, True])
def test_identity_probes_give_the_exact_trace(is_complex):
    A = matrices.anderson(5, 3, 4.0, 3, is_complex)
    lam0 = np.linalg.eigvalsh(A.to_dense())
    a, b = _gap_interval(lam0, 50, 9)
    lam, U, l1, l2, coef = _setup(A, a, b, 120)
    exact = float(np.sum(_rho_direct(coef, l1 * lam + l2)))
    # the n basis vectors sum to I (rather than averaging to it): n times the mean
    est = A.n * trace.trace_estimate(A.to_scipy(), coef, l1, l2, np.eye(A.n))
    assert abs(est - exact) <= 1e-10 * max(1.0, abs(exact))


def test_all_sign_vectors_are_unbiased():
    """Over every sign vector of length n, E[z z^T] = I exactly, so the mean
    of z^T M z is tr M (brute force on n = 8)."""
    A = matrices.random_sparse_hermitian(8, 3, 5, False)
    lam = np.linalg.eigvalsh(A.to_dense())
    lam_s, U, l1, l2, coef = _setup(A, lam[2] - 1e-3, lam[5] + 1e-3, 30)
    Z = np.array(list(itertools.product([-1.0, 1.0], repeat=8))).T  # 8 x 256
    est = trace.trace_estimate(A.to_scipy(), coef, l1, l2, Z)
    exact = float(np.sum(_rho_direct(coef, l1 * lam_s + l2)))
    assert abs(est - exact) <= 1e-11 * max(1.0, abs(exact))


@pytest.mark.parametrize("is_complex", [False, True])
def test_random_probes_within_six_sigma(is_complex):
    A = matrices.anderson(6, 3, 5.0, 9, is_complex)
    lam0 = np.linalg.eigvalsh(A.to_dense())
    a, b = _gap_interval(lam0, 80, 12)
    lam, U, l1, l2, coef = _setup(A, a, b, 200)
    r = _rho_direct(coef, l1 * lam + l2)
    M = (U * r) @ U.conj().T
    exact = float(np.real(np.trace(M)))
    m = 32
    off = np.real(M) - np.diag(np.diag(np.real(M)))
    sigma = math.sqrt(2.0 * np.sum(off ** 2) / m)  # real +-1 probes: Var(z^T M z) = 2 sum_{i!=j} Re(M_ij)^2
    Z = rng.rademacher_block(17, rng.STREAM_TRACE, A.n, m)
    est = trace.trace_estimate(A.to_scipy(), coef, l1, l2, Z)
    assert abs(est - exact) <= 6.0 * sigma
    # a sharp filter with its ends in gaps counts the eigenvalues inside
    assert abs(exact - 12) < 0.5


def test_rademacher_block_layout():
    Z = rng.rademacher_block(4, rng.STREAM_TRACE, 7, 5)
    assert Z.shape == (7, 5) and set(np.unique(Z)) <= {-1.0, 1.0}
    top = rng.raw64(4, rng.STREAM_TRACE, np.arange(35, dtype=np.uint64)) >> np.uint64(63)
    assert np.array_equal(Z.ravel(), np.where(top == 0, -1.0, 1.0))
    big = rng.rademacher_block(4, rng.STREAM_TRACE, 1000, 10)
    assert abs(big.mean()) < 0.05


def test_subspace_size_rule():
    assert trace.subspace_size(10.0, 1.8, 1000, 1024) == 18
    assert trace.subspace_size(10.2, 1.8, 1000, 1024) == 19   # ceil(18.36)
    assert trace.subspace_size(-3.0, 1.8, 1000, 1024) == 2    # floored at e~ = 1
    assert trace.subspace_size(900.0, 1.8, 1000, 1024) == 1000
    assert trace.subspace_size(900.0, 1.8, 5000, 1024) == 1024


def test_moments_give_the_trace_estimate_and_the_exact_trace():
    """sum_j a_j mu_j is the same Hutchinson estimate as trace_estimate (same
    probes), and with the identity as the probe block it is the exact trace
    sum_i rho(l(lambda_i)) from a dense eigendecomposition."""
    import numpy as np
    from oracle import chebyshev as cb
    from oracle import fsi, trace
    from synth import matrices, rng
    A = matrices.anderson(7, 3, 3.0, 5, True)
    As = A.to_scipy()
    lmin, lmax = fsi.gershgorin(As)
    l1, l2 = cb.linear_map(lmin, lmax)
    k = 120
    coef = cb.filter_coefficients(l1 * -0.4 + l2, l1 * 0.9 + l2, k)
    Z = rng.rademacher_block(3, rng.STREAM_TEST, A.n, 8)
    mu = trace.chebyshev_trace_moments(As, l1, l2, Z, k)
    assert abs(coef @ mu - trace.trace_estimate(As, coef, l1, l2, Z)) < 1e-9 * A.n
    mu_exact = trace.chebyshev_trace_moments(As, l1, l2, np.eye(A.n), k) * A.n
    lam = np.linalg.eigvalsh(A.to_dense())
    th = np.arccos(np.clip(l1 * lam + l2, -1, 1))
    for j in (0, 1, 2, 17, k):
        assert abs(mu_exact[j] - np.sum(np.cos(j * th))) < 1e-8 * A.n
    assert abs(coef @ mu_exact - np.sum(cb.cheb_direct(coef, l1 * lam + l2))) < 1e-8 * A.n
