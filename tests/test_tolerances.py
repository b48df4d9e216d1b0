"""The Alg. 2 parity tolerance (gpu_util.clenshaw_tol) is neither loose nor
tight: an FP32 evaluation of the recurrence in another summation order (numpy
float32 / complex64, FP32 matrix values, FP32 accumulation) stays 8 times
inside it, and dropping any single term a_j T_j(A_hat) Y of the oracle's
expansion (a mistake planted on the CPU, in the oracle's input) moves the
result by more than 10 times the tolerance."""
import numpy as np
import pytest
import scipy.sparse as sp

from gpu_util import EPS32, clenshaw_tol
from oracle import chebyshev as cb
from oracle import fsi
from oracle.filter import clenshaw_apply
from synth import matrices, rng, workloads

CASES = [
    ("lap2d_32", lambda: workloads.lap2d_32().matrix(), 24),
    ("anderson_c_10", lambda: matrices.anderson(10, 3, 4.0, 7, True), 37),
    ("random_c_777", lambda: matrices.random_sparse_hermitian(777, 6, 3, True), 13),
]


def _f32_clenshaw(As, coef, l1, l2, X, is_complex):
    """Alg. 2 with every operation in single precision (test helper only)."""
    lo = np.complex64 if is_complex else np.float32
    Ah = (l1 * As + l2 * sp.identity(As.shape[0])).astype(lo).tocsr()
    Y = X.astype(lo)
    c = coef.astype(np.float32)
    k = len(coef) - 1
    b1, b2 = c[k] * Y, np.zeros_like(Y)
    for j in range(k - 1, 0, -1):
        b1, b2 = np.float32(2) * (Ah @ b1) - b2 + c[j] * Y, b1
    return Ah @ b1 - b2 + c[0] * Y


@pytest.mark.parametrize("name,make,p", CASES)
def test_fp32_tolerance_between_rounding_and_a_dropped_term(name, make, p):
    A = make()
    As = A.to_scipy()
    lmin, lmax = fsi.gershgorin(As)
    l1, l2 = cb.linear_map(lmin, lmax)
    coef = cb.filter_coefficients(-0.1, 0.05, 150)   # the FP32 parity filter of test_gpu_steps
    X = rng.uniform_block(7, rng.STREAM_TEST, A.n, p, A.is_complex)
    ref = clenshaw_apply(As, coef, l1, l2, X)
    tol = clenshaw_tol(coef, X, EPS32)
    err = np.max(np.abs(_f32_clenshaw(As, coef, l1, l2, X, A.is_complex) - ref))
    assert err * 8 <= tol, (err, tol)
    k = len(coef) - 1
    for j in (0, 1, k // 4, k // 2, 3 * k // 4, k - 1, k):
        bad = coef.copy()
        bad[j] = 0.0
        diff = np.max(np.abs(clenshaw_apply(As, bad, l1, l2, X) - ref))
        assert diff > 10 * tol, (j, coef[j], diff, tol)
