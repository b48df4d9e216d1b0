"""The dense products of Alg. 4 on the tcgen05 tensor cores: the Gram product
X^H Y (apf_gram_tc) and the tall block update Z = beta Z0 + alpha X M
(apf_block_update).  Both cut FP64 values into seven 8-bit digits held in
bf16, accumulate the digit products exactly (FP32 in TMEM per 32-row chunk,
then 32- and 64-bit integers) and round once to FP64.  Checked against the
FP64 product and the definition, and through whole solves that use them for
CholQR and Rayleigh-Ritz."""
import numpy as np
import pytest

from gpu_util import EPS64, dev, empty_like_np, host
from synth import matrices, rng

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


def _tol(n, X, Y):
    """Error bound of the slicing: about n 2^-55 relative to 2^(e_a + e_b),
    with 2^e_a < 2 max |x_a|; a factor 8 of slack."""
    return 8.0 * n * EPS64 * np.max(np.abs(X)) * np.max(np.abs(Y))


@pytest.mark.parametrize("is_complex", [False, True])
@pytest.mark.parametrize("n,pa,pb", [(1000, 37, 45), (64, 1, 1), (3001, 64, 33), (257, 100, 100),
                                     (20000, 160, 160), (5003, 200, 7)])
def test_gram_tc_matches_fp64_and_definition(B, ctx, is_complex, n, pa, pb):
    X = rng.uniform_block(50 + pa, rng.STREAM_TEST, n, pa, is_complex)
    Y = rng.uniform_block(60 + pb, rng.STREAM_TEST, n, pb, is_complex)
    ref = X.conj().T @ Y
    G = empty_like_np((pa, pb), is_complex)
    B.gram_tc(ctx, dev(X), dev(Y), G)
    G64 = empty_like_np((pa, pb), is_complex)
    B.gram(ctx, dev(X), dev(Y), G64)
    tol = _tol(n, X, Y)
    assert np.max(np.abs(host(G) - ref)) <= tol
    assert np.max(np.abs(host(G) - host(G64))) <= tol + 4 * n * EPS64


@pytest.mark.parametrize("is_complex", [False, True])
def test_gram_tc_columns_of_very_different_size(B, ctx, is_complex):
    """Each column has its own power of two: columns 1e-30 .. 1e30 apart keep
    their relative accuracy (entry (a, b) relative to max|x_a| max|y_b|)."""
    n, p = 4000, 24
    X = rng.uniform_block(7, rng.STREAM_TEST, n, p, is_complex) * np.logspace(-30, 30, p)
    Y = rng.uniform_block(8, rng.STREAM_TEST, n, p, is_complex) * np.logspace(30, -30, p)
    ref = X.conj().T @ Y
    G = empty_like_np((p, p), is_complex)
    B.gram_tc(ctx, dev(X), dev(Y), G)
    scale = np.outer(np.max(np.abs(X), axis=0), np.max(np.abs(Y), axis=0))
    assert np.max(np.abs(host(G) - ref) / scale) <= 8.0 * n * EPS64


def test_gram_tc_same_block_twice(B, ctx):
    """X^H X with X passed as both operands (one set of slices): Hermitian to
    rounding and equal to the definition."""
    X = rng.uniform_block(9, rng.STREAM_TEST, 9000, 96, True)
    Xd = dev(X)
    G = empty_like_np((96, 96), True)
    B.gram_tc(ctx, Xd, Xd, G)
    g = host(G)
    assert np.max(np.abs(g - X.conj().T @ X)) <= _tol(9000, X, X)
    assert np.max(np.abs(g - g.conj().T)) <= _tol(9000, X, X)


@pytest.mark.parametrize("prec", ["F64", "F32_DEFECT"])
@pytest.mark.parametrize("is_complex", [False, True])
def test_solve_with_tensor_core_grams(B, ctx, prec, is_complex):
    """CholQR and Rayleigh-Ritz on tensor-core Grams: the same eigenvalues as
    the definition, residuals at 1e-10, orthonormal vectors."""
    A = matrices.anderson(10, 3, 5.0, 61, is_complex)
    lam = np.linalg.eigvalsh(A.to_dense())
    i, c = 480, 12
    a, b = 0.5 * (lam[i - 1] + lam[i]), 0.5 * (lam[i + c - 1] + lam[i + c])
    M = B.Matrix.from_csr(ctx, A.n, A.rowptr, A.colidx, A.vals)
    r = B.solve(ctx, M, B.default_params(a=a, b=b, p=24, seed=2, gram_tensor_cores=1,
                                         filter_precision=getattr(B, "APF_FILTER_" + prec)))
    r0 = B.solve(ctx, M, B.default_params(a=a, b=b, p=24, seed=2, gram_tensor_cores=0,
                                          filter_precision=getattr(B, "APF_FILTER_" + prec)))
    got0 = r0.eigvals()
    r0.close()
    assert np.max(np.abs(got0 - lam[i:i + c])) <= 1e-10 * np.abs(lam).max()  # the FP64-core form
    got, V, st = r.eigvals(), r.eigvecs(A.n, A.is_complex), r.stats()
    r.close()
    M.close()
    assert got.size == c
    assert np.max(np.abs(got - lam[i:i + c])) <= 1e-10 * np.abs(lam).max()
    res = np.linalg.norm(A.to_scipy() @ V - V * got, axis=0)
    assert res.max() <= 1e-10 * st["norm_a"]  # norm_a <= ||A||: conservative
    assert np.max(np.abs(V.conj().T @ V - np.eye(c))) < 1e-10


def test_gram_tc_rejects_bad_arguments(B, ctx):
    import torch
    X = torch.zeros((10, 4), dtype=torch.float64, device="cuda")
    lib = B.Library.load()
    G = torch.zeros((4, 4), dtype=torch.float64, device="cuda")
    assert lib.apf_gram_tc(ctx.h, 99, 10, 4, 4, X.data_ptr(), 4, X.data_ptr(), 4, G.data_ptr(), 4) == B.APF_ERR_ARG
    assert lib.apf_gram_tc(ctx.h, B.APF_R64, 10, 4, 4, X.data_ptr(), 3, X.data_ptr(), 4, G.data_ptr(), 4) == \
        B.APF_ERR_ARG
    big = torch.zeros((2, 1100), dtype=torch.float64, device="cuda")
    Gb = torch.zeros((1100, 1100), dtype=torch.float64, device="cuda")
    assert lib.apf_gram_tc(ctx.h, B.APF_R64, 2, 1100, 1100, big.data_ptr(), 1100, big.data_ptr(), 1100,
                           Gb.data_ptr(), 1100) == B.APF_ERR_ARG


@pytest.mark.parametrize("is_complex", [False, True])
@pytest.mark.parametrize("n,pa,pb", [(1000, 37, 45), (129, 1, 1), (3001, 160, 33), (20000, 300, 300),
                                     (777, 200, 7)])
def test_block_update_tc_matches_fp64(B, ctx, is_complex, n, pa, pb):
    """Z = beta Z + alpha X M on the tensor cores against the FP64 cores and
    numpy: rows of X and columns of M carry their own powers of two, so the
    error is about pa 2^-55 max|x_i| max|m_j| per entry."""
    X = rng.uniform_block(70 + pa, rng.STREAM_TEST, n, pa, is_complex) * np.logspace(-3, 3, n)[:, None]
    M = rng.uniform_block(80 + pb, rng.STREAM_TEST, pa, pb, is_complex)
    Z0 = rng.uniform_block(90, rng.STREAM_TEST, n, pb, is_complex)
    for alpha, beta in ((1.0, 0.0), (-1.0, 1.0)):
        ref = beta * Z0 + alpha * (X @ M)
        Zt = dev(Z0.copy())
        B.block_update(ctx, dev(X), dev(M), Zt, alpha, beta, tensor_cores=True)
        Zf = dev(Z0.copy())
        B.block_update(ctx, dev(X), dev(M), Zf, alpha, beta, tensor_cores=False)
        scale = np.outer(np.max(np.abs(X), axis=1), np.max(np.abs(M), axis=0))
        tol = 8.0 * pa * EPS64 * scale + 4 * EPS64 * np.abs(ref)
        assert np.all(np.abs(host(Zt) - ref) <= tol)
        assert np.all(np.abs(host(Zt) - host(Zf)) <= tol + 8.0 * pa * EPS64 * scale)
