"""One outer iteration of Alg. 4 at full size, GPU against the oracle, element
by element: the 64^3 complex Anderson workload (n = 262,144, p = 160) and the
96^3 Kohn-Sham-like one (n = 884,736, p = 300).

From the same seeded block X0 and the same map l (Gershgorin bounds), both
sides apply the FP64 filter of fixed degree 40 (Alg. 2), orthonormalise by
CholQR2, run Rayleigh-Ritz (Alg. 1) and compute the residual norms.  The
filtered block must agree within the Alg. 2 bound, the Ritz values and the
residual norms within 1e-10 ||A|| (||A|| from the oracle's Lanczos Ritz
values).  The oracle's filter runs column-parallel (tests/oracle_pool.py,
identical to one call); its CholQR2 and Rayleigh-Ritz run on the whole block.
"""
import numpy as np
import pytest

from gpu_util import EPS64, clenshaw_tol, dev, empty_like_np, host
from oracle import chebyshev as cb
from oracle import fsi
from oracle_pool import clenshaw_apply_parallel
from synth import rng, workloads

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

DEGREE = 40


@pytest.fixture(scope="module")
def B(gpu_lib):
    from paper_2604_00914_gb300 import binding
    return binding


@pytest.mark.parametrize("name", ["anderson3d_c_64", "ks8_96"])
def test_one_outer_iteration_matches_oracle(B, name):
    import torch
    w = workloads.WORKLOADS[name]()
    A = w.matrix()
    As = A.to_scipy()
    lmin, lmax = fsi.gershgorin(As)
    l1, l2 = cb.linear_map(lmin, lmax)
    coef = cb.filter_coefficients(l1 * w.a + l2, l1 * w.b + l2, DEGREE)
    X0 = rng.uniform_block(w.seed, rng.STREAM_INIT_BLOCK, A.n, w.p, A.is_complex)
    v0 = rng.uniform_block(w.seed, rng.STREAM_LANCZOS, A.n, 1, A.is_complex)[:, 0]
    _, _, info = fsi.lanczos_bounds(As, 40, v0)
    normA = max(abs(info["theta_min"]), abs(info["theta_max"]))

    # oracle: Alg. 2, CholQR2, Alg. 1, residuals
    X_ref = clenshaw_apply_parallel(A, coef, l1, l2, X0)
    Q_ref = fsi.cholqr2(X_ref)
    lam_ref, V_ref = fsi.rayleigh_ritz(As, Q_ref)
    res_ref = fsi.residual_norms(As, V_ref, lam_ref)
    del Q_ref, V_ref

    ctx = B.Context(0)
    try:
        M = B.Matrix.from_csr(ctx, A.n, A.rowptr, A.colidx, A.vals)
        X = empty_like_np((A.n, w.p), A.is_complex)
        B.filter_apply(ctx, M, coef, l1, l2, dev(X0), X, B.APF_FILTER_F64)
        assert np.max(np.abs(host(X) - X_ref)) <= clenshaw_tol(coef, X0, EPS64)
        del X_ref
        B.cholqr2(ctx, X)
        lam = torch.zeros(w.p, dtype=torch.float64, device="cuda")
        V = torch.empty_like(X)
        B.rayleigh_ritz(ctx, M, X, lam, V)
        res = B.residual_norms(ctx, M, V, lam)
        lam = host(lam)
        M.close()
    finally:
        ctx.close()
    assert np.max(np.abs(lam - lam_ref)) <= 1e-10 * normA, np.max(np.abs(lam - lam_ref)) / normA
    assert np.max(np.abs(res - res_ref)) <= 1e-10 * normA, np.max(np.abs(res - res_ref)) / normA
