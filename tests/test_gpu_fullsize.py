"""The bench configuration at full size (64^3 complex Anderson, n = 262,144,
p = 160, FP32 defect filter): properties that hold at any size, checked on the
host in FP64, and sampled comparisons with the oracle.

The dense definition is out of reach at this size, so:
 - every returned pair has ||A v - lambda v|| <= 1e-10 ||A||_est, recomputed here
   with scipy in FP64; the vectors are orthonormal; all values lie in [a, b];
 - a second solve from a different random start (and a larger subspace) finds
   the same eigenvalues: a missed eigenvalue would have to be missed twice;
 - the count agrees with the kernel-polynomial estimate of the workload (98.9);
 - four Clenshaw steps on the full matrix and block match the oracle's Alg. 2.
"""
import numpy as np
import pytest

from gpu_util import EPS32, clenshaw_tol, dev, empty_like_np, host
from oracle import chebyshev as cb
from oracle.filter import clenshaw_apply
from synth import rng, workloads

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


@pytest.fixture(scope="module")
def B(gpu_lib):
    from paper_2604_00914_gb300 import binding
    return binding


@pytest.fixture(scope="module")
def setup(B):
    w = workloads.anderson3d_c_64()
    A = w.matrix()
    ctx = B.Context(0)
    M = B.Matrix.from_csr(ctx, A.n, A.rowptr, A.colidx, A.vals)
    yield w, A, ctx, M
    ctx.close()


def _solve(B, ctx, M, A, **kw):
    r = B.solve(ctx, M, B.default_params(**kw))
    out = dict(lam=r.eigvals(), V=r.eigvecs(A.n, True), stats=r.stats())
    r.close()
    return out


def test_full_size_solve_properties_and_repeatability(B, setup):
    w, A, ctx, M = setup
    one = _solve(B, ctx, M, A, a=w.a, b=w.b, p=w.p, seed=w.seed, filter_precision=B.APF_FILTER_F32_DEFECT)
    lam, V, st = one["lam"], one["V"], one["stats"]
    assert 90 <= lam.size <= 110          # kernel-polynomial estimate: 98.9
    assert np.all((lam >= w.a) & (lam <= w.b))
    res = np.linalg.norm(A.to_scipy() @ V - V * lam, axis=0)
    assert res.max() <= 1e-10 * st["norm_a"]  # norm_a <= ||A||: conservative
    assert np.max(np.abs(V.conj().T @ V - np.eye(lam.size))) < 1e-10
    two = _solve(B, ctx, M, A, a=w.a, b=w.b, p=w.p + 20, seed=w.seed + 77,
                 filter_precision=B.APF_FILTER_F32_DEFECT)
    assert two["lam"].size == lam.size
    assert np.max(np.abs(two["lam"] - lam)) <= 1e-10 * st["norm_a"]


def test_full_size_filter_steps_match_oracle(B, setup):
    w, A, ctx, M = setup
    lmin, lmax = -5.6, 5.6
    l1, l2 = cb.linear_map(lmin, lmax)
    coef = cb.filter_coefficients(l1 * w.a + l2, l1 * w.b + l2, 4)
    X = rng.uniform_block(w.seed, rng.STREAM_TEST, A.n, w.p, True)
    Y = empty_like_np((A.n, w.p), True)
    B.filter_apply(ctx, M, coef, l1, l2, dev(X), Y, B.APF_FILTER_F32)
    ref = clenshaw_apply(A.to_scipy(), coef, l1, l2, X)
    assert np.max(np.abs(host(Y) - ref)) <= clenshaw_tol(coef, X, EPS32)
