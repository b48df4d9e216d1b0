"""GPU parity of each step of the path against the oracle, through the C ABI.

Sizes span several tiles and ragged tails: n up to a few thousand, block
widths that are not multiples of the 16-byte vector or the 32-wide tiles.
"""
import numpy as np
import pytest

from gpu_util import EPS32, EPS64, clenshaw_tol, dev, empty_like_np, host
from oracle import chebyshev as cb
from oracle import fsi
from oracle.filter import clenshaw_apply
from synth import matrices, rng, workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B(gpu_lib):
    from paper_2604_00914_gb300 import binding
    return binding


@pytest.fixture(scope="module")
def ctx(B):
    c = B.Context(0)
    yield c
    c.close()


def _mat(B, ctx, A):
    return B.Matrix.from_csr(ctx, A.n, A.rowptr, A.colidx, A.vals)


CASES = [
    ("lap2d_32", lambda: workloads.lap2d_32().matrix(), 24),
    ("anderson_c_10", lambda: matrices.anderson(10, 3, 4.0, 7, True), 37),
    ("random_c_777", lambda: matrices.random_sparse_hermitian(777, 6, 3, True), 13),
    ("random_r_1500", lambda: matrices.random_sparse_hermitian(1500, 9, 4, False), 61),
    ("ks8_10", lambda: matrices.ks_like_3d(10, 2, n_wells=5), 5),
]


@pytest.mark.parametrize("is_complex", [False, True])
def test_random_block_matches_generator_bitwise(B, ctx, is_complex):
    """The device SplitMix64 block equals synth.rng's, bit for bit."""
    n, p = 1001, 19
    X = empty_like_np((n, p), is_complex)
    B.random_block(ctx, 20260405, 1, X)
    ref = rng.uniform_block(20260405, 1, n, p, is_complex)
    assert np.array_equal(host(X), ref)


@pytest.mark.parametrize("name,make,p", CASES)
def test_spmm_matches_scipy(B, ctx, name, make, p):
    A = make()
    M = _mat(B, ctx, A)
    X = rng.uniform_block(5, rng.STREAM_TEST, A.n, p, A.is_complex)
    Y = empty_like_np((A.n, p), A.is_complex)
    B.spmm(ctx, M, dev(X), Y)
    ref = A.to_scipy() @ X
    assert np.max(np.abs(host(Y) - ref)) <= 64 * EPS64 * np.max(np.abs(ref)) * 30


@pytest.mark.parametrize("name,make,p", CASES)
@pytest.mark.parametrize("k,damp", [(0, cb.DAMP_LANCZOS_M), (1, cb.DAMP_LANCZOS_M), (2, cb.DAMP_JACKSON),
                                    (40, cb.DAMP_JACKSON), (271, cb.DAMP_LANCZOS_M)])
def test_filter_f64_matches_oracle(B, ctx, name, make, p, k, damp):
    """Alg. 2 in FP64 on the GPU against the oracle's Alg. 2."""
    A = make()
    As = A.to_scipy()
    M = _mat(B, ctx, A)
    lmin, lmax = fsi.gershgorin(As)
    l1, l2 = cb.linear_map(lmin, lmax)
    mid = 0.5 * (lmin + lmax)
    am, bm = l1 * (mid - 0.3) + l2, l1 * (mid + 0.2) + l2
    coef = cb.filter_coefficients(am, bm, max(k, 1), damp)[:k + 1]
    X = rng.uniform_block(6, rng.STREAM_TEST, A.n, p, A.is_complex)
    Y = empty_like_np((A.n, p), A.is_complex)
    B.filter_apply(ctx, M, coef, l1, l2, dev(X), Y, B.APF_FILTER_F64)
    ref = clenshaw_apply(As, coef, l1, l2, X)
    assert np.max(np.abs(host(Y) - ref)) <= clenshaw_tol(coef, X, EPS64)


@pytest.mark.parametrize("name,make,p", CASES[:3])
def test_filter_f32_matches_oracle(B, ctx, name, make, p):
    A = make()
    As = A.to_scipy()
    M = _mat(B, ctx, A)
    lmin, lmax = fsi.gershgorin(As)
    l1, l2 = cb.linear_map(lmin, lmax)
    coef = cb.filter_coefficients(-0.1, 0.05, 150)
    X = rng.uniform_block(7, rng.STREAM_TEST, A.n, p, A.is_complex)
    Y = empty_like_np((A.n, p), A.is_complex)
    B.filter_apply(ctx, M, coef, l1, l2, dev(X), Y, B.APF_FILTER_F32)
    ref = clenshaw_apply(As, coef, l1, l2, X)
    err = np.max(np.abs(host(Y) - ref))
    assert err <= clenshaw_tol(coef, X, EPS32)
    assert err > 1e-12  # it really ran in single precision


@pytest.mark.parametrize("name,make,p", CASES[:3])
def test_filter_defect_matches_oracle(B, ctx, name, make, p):
    """Defect form: rho(A)V = V rho(lam) + D with D from an FP32 recurrence
    driven by R = AV - V lam.  For near-eigenvectors the error scales with ||R||:
    here V = exact eigenvectors + 1e-6 noise, so the FP32 error is ~1e-6 times
    the plain FP32 error."""
    A = make()
    As = A.to_scipy()
    Ad = A.to_dense()
    M = _mat(B, ctx, A)
    lam_all, U = np.linalg.eigh(Ad)
    lmin, lmax = lam_all[0] - 0.05, lam_all[-1] + 0.05
    l1, l2 = cb.linear_map(lmin, lmax)
    mid = 0.5 * (lmin + lmax)
    coef = cb.filter_coefficients(l1 * (mid - 0.3) + l2, l1 * (mid + 0.25) + l2, 200)
    sel = np.arange(0, A.n, max(1, A.n // p))[:p]
    noise = rng.uniform_block(8, rng.STREAM_TEST, A.n, p, A.is_complex)
    V = U[:, sel] + 1e-6 * noise
    AV = As @ V
    lam = np.real(np.sum(V.conj() * AV, axis=0) / np.sum(V.conj() * V, axis=0))
    Y = empty_like_np((A.n, p), A.is_complex)
    B.filter_apply_defect(ctx, M, coef, l1, l2, dev(V), dev(AV), dev(lam), Y)
    ref = clenshaw_apply(As, coef, l1, l2, V)
    R = AV - V * lam
    tol = clenshaw_tol(coef, l1 * R, EPS32) + clenshaw_tol(coef, V, EPS64)
    err = np.max(np.abs(host(Y) - ref))
    assert err <= tol, (err, tol)
    assert err < 1e-9


@pytest.mark.parametrize("is_complex", [False, True])
@pytest.mark.parametrize("n,pa,pb", [(1000, 37, 45), (64, 1, 1), (3001, 64, 33), (257, 100, 100)])
def test_gram_matches_definition(B, ctx, is_complex, n, pa, pb):
    X = rng.uniform_block(9, rng.STREAM_TEST, n, pa, is_complex)
    Y = rng.uniform_block(10, rng.STREAM_TEST, n, pb, is_complex)
    G = empty_like_np((pa, pb), is_complex)
    B.gram(ctx, dev(X), dev(Y), G)
    ref = X.conj().T @ Y
    assert np.max(np.abs(host(G) - ref)) <= 4 * n * EPS64 * 1.0


@pytest.mark.parametrize("is_complex", [False, True])
@pytest.mark.parametrize("kappa", [1e2, 1e7, 1e11])
def test_cholqr2(B, ctx, is_complex, kappa):
    n, p = 2000, 29
    G = rng.uniform_block(3, rng.STREAM_TEST, n, p, is_complex)
    Q0, _ = np.linalg.qr(G)
    W, _ = np.linalg.qr(rng.uniform_block(4, rng.STREAM_TEST, p, p, is_complex))
    X = Q0 @ np.diag(np.logspace(0, -np.log10(kappa), p)) @ W
    Xd = dev(X)
    B.cholqr2(ctx, Xd)
    Q = host(Xd)
    assert np.max(np.abs(Q.conj().T @ Q - np.eye(p))) < 1e-13
    assert np.linalg.norm(X - Q @ (Q.conj().T @ X)) < 1e-10 * np.linalg.norm(X)
    ref = fsi.cholqr2(X)
    # the same R-factor sign convention (positive diagonal) gives the same Q
    assert np.max(np.abs(Q - ref)) < 1e-6 * kappa ** 0.5


def _herm(p, seed, is_complex):
    M = rng.uniform_block(seed, rng.STREAM_TEST, p, p, is_complex)
    return 0.5 * (M + M.conj().T)


@pytest.mark.parametrize("is_complex", [False, True])
@pytest.mark.parametrize("p", [1, 2, 3, 24, 37, 160])
def test_eigh_small_matches_lapack(B, ctx, is_complex, p):
    Bm = _herm(p, 11 + p, is_complex)
    w = empty_like_np((p,), False)
    U = empty_like_np((p, p), is_complex)
    B.eigh_small(ctx, dev(Bm), w, U)
    ref = np.linalg.eigvalsh(Bm)
    wh, Uh = host(w), host(U)
    scale = max(1.0, np.abs(ref).max())
    assert np.max(np.abs(wh - ref)) <= 50 * p * EPS64 * scale
    assert np.max(np.abs(Uh.conj().T @ Uh - np.eye(p))) <= 50 * p * EPS64
    assert np.max(np.abs(Bm @ Uh - Uh * wh)) <= 100 * p * EPS64 * scale


@pytest.mark.parametrize("is_complex", [False, True])
def test_eigh_small_degenerate_and_zero(B, ctx, is_complex):
    p = 16
    for Bm in (np.zeros((p, p)), np.eye(p), np.diag(np.repeat([1.0, -2.0, 3.0, 3.0], 4))):
        Bm = Bm.astype(np.complex128 if is_complex else np.float64)
        w = empty_like_np((p,), False)
        U = empty_like_np((p, p), is_complex)
        B.eigh_small(ctx, dev(Bm), w, U)
        wh, Uh = host(w), host(U)
        assert np.allclose(wh, np.linalg.eigvalsh(Bm), atol=1e-14)
        assert np.max(np.abs(Uh.conj().T @ Uh - np.eye(p))) < 1e-13
        assert np.max(np.abs(Bm @ Uh - Uh * wh)) < 1e-13


@pytest.mark.parametrize("name,make,p", CASES[:4])
def test_rayleigh_ritz_and_residuals(B, ctx, name, make, p):
    A = make()
    As = A.to_scipy()
    M = _mat(B, ctx, A)
    X = rng.uniform_block(12, rng.STREAM_TEST, A.n, p, A.is_complex)
    Q = fsi.cholqr2(X)
    w = empty_like_np((p,), False)
    V = empty_like_np((A.n, p), A.is_complex)
    B.rayleigh_ritz(ctx, M, dev(Q), w, V)
    lam_ref, V_ref = fsi.rayleigh_ritz(As, Q)
    normA = np.abs(fsi.gershgorin(As)).max()
    assert np.max(np.abs(host(w) - lam_ref)) <= 1e3 * EPS64 * normA
    res = B.residual_norms(ctx, M, V, w)
    res_ref = fsi.residual_norms(As, host(V), host(w))
    assert np.max(np.abs(res - res_ref)) <= 1e3 * EPS64 * normA


@pytest.mark.parametrize("name,make,p", CASES)
def test_spectrum_bounds_match_oracle(B, ctx, name, make, p):
    A = make()
    As = A.to_scipy()
    M = _mat(B, ctx, A)
    seed = 20260431
    out = B.spectrum_bounds(ctx, M, 40, seed, 0.01)
    v0 = rng.uniform_block(seed, rng.STREAM_LANCZOS, A.n, 1, A.is_complex)[:, 0]
    lmin, lmax, info = fsi.lanczos_bounds(As, 40, v0, 0.01)
    g = fsi.gershgorin(As)
    span = g[1] - g[0]
    assert abs(out[4] - g[0]) <= 1e-13 * span and abs(out[5] - g[1]) <= 1e-13 * span
    assert abs(out[2] - info["theta_min"]) <= 1e-9 * span
    assert abs(out[3] - info["theta_max"]) <= 1e-9 * span
    assert abs(out[0] - lmin) <= 1e-7 * span and abs(out[1] - lmax) <= 1e-7 * span
    lam = np.linalg.eigvalsh(A.to_dense())
    assert out[0] <= lam[0] and out[1] >= lam[-1]
