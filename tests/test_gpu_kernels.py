"""Every compiled variant of the FP32 Clenshaw step (Alg. 2) gives the same
bits: SELL-8 one step per launch in each (G, VPT) shape, SELL-8 two steps per
pass over the reverse Cuthill-McKee copy, SELL-8 in column tiles of each
compiled tile width (also on blocks wider than 1024 columns), the same with
the near rows of W staged in shared memory, and CSR.  The autotuner picks among
them by time, so a result must not depend on the pick (a serving request gives
the same answer alone and in a mix).  Matrices with a wide natural bandwidth
(periodic lattices) get the permuted copy; small ones stay in natural order.
"""
import numpy as np
import pytest

from gpu_util import EPS32, clenshaw_tol, dev, empty_like_np, host
from oracle import chebyshev as cb
from oracle import fsi
from oracle.filter import clenshaw_apply
from synth import matrices, rng, workloads

pytestmark = pytest.mark.gpu

SELL_SHAPES = [(8, 1), (8, 2), (8, 3), (8, 4), (16, 2), (16, 3), (16, 4), (16, 5), (16, 6),
               (32, 2), (32, 3), (32, 4), (32, 5), (32, 6), (32, 8)]
CT_SHAPES = [(8, 1), (8, 2), (16, 1), (8, 4), (16, 2), (32, 1), (16, 4), (32, 2)]

MATS = [
    ("lap2d_32", lambda: workloads.lap2d_32().matrix()),                      # natural order
    ("anderson_r_17_periodic", lambda: matrices.anderson(17, 3, 3.5, 5, False)),  # RCM copy
    ("anderson_c_70_2d", lambda: matrices.anderson(70, 2, 2.0, 6, True)),     # RCM copy
    ("ks_like_12", lambda: matrices.ks_like_3d(12, 3, n_wells=6)),            # near rows +-4
]


@pytest.fixture(scope="module")
def B(gpu_lib):
    from paper_2604_00914_gb300 import binding
    return binding


@pytest.fixture(scope="module")
def ctx(B):
    c = B.Context(0)
    yield c
    c.close()


def _variants(p, is_complex):
    E = 2 if is_complex else 4
    nvec = -(-p // E)
    out = [(3, 0, 0)]
    for kind in (1, 2):
        out += [(kind, g, v) for g, v in SELL_SHAPES if g * v >= nvec]
    out += [(kind, g, v) for kind in (4, 5) for g, v in CT_SHAPES]
    return out


@pytest.mark.parametrize("name,make", MATS)
@pytest.mark.parametrize("p", [5, 24, 37, 140])
def test_all_step_kernels_agree_bitwise(B, ctx, name, make, p):
    A = make()
    As = A.to_scipy()
    lmin, lmax = fsi.gershgorin(As)
    l1, l2 = cb.linear_map(lmin, lmax)
    coef = cb.filter_coefficients(-0.12, 0.02, 121)
    X = rng.uniform_block(11, rng.STREAM_TEST, A.n, p, A.is_complex)
    ref = clenshaw_apply(As, coef, l1, l2, X)
    tol = clenshaw_tol(coef, X, EPS32)
    M = B.Matrix.from_csr(ctx, A.n, A.rowptr, A.colidx, A.vals)
    first = None
    for kind, g, v in _variants(p, A.is_complex):
        M.set_filter_kernel(kind, g, v)
        Y = empty_like_np((A.n, p), A.is_complex)
        B.filter_apply(ctx, M, coef, l1, l2, dev(X), Y, B.APF_FILTER_F32)
        y = host(Y)
        assert np.max(np.abs(y - ref)) <= tol, (kind, g, v)
        if first is None:
            first = y
        else:
            assert np.array_equal(first, y), (kind, g, v, np.max(np.abs(first - y)))
    M.close()


@pytest.mark.parametrize("name,make", MATS[1:])
def test_defect_form_agrees_across_kernels(B, ctx, name, make):
    A = make()
    As = A.to_scipy()
    p = 24
    lmin, lmax = fsi.gershgorin(As)
    l1, l2 = cb.linear_map(lmin, lmax)
    coef = cb.filter_coefficients(-0.12, 0.02, 121)
    V, _ = np.linalg.qr(rng.uniform_block(12, rng.STREAM_TEST, A.n, p, A.is_complex))
    V = np.ascontiguousarray(V)
    AV = As @ V
    lam = np.real(np.sum(V.conj() * AV, axis=0))
    M = B.Matrix.from_csr(ctx, A.n, A.rowptr, A.colidx, A.vals)
    outs = []
    for kind, g, v in [(3, 0, 0), (1, 0, 0), (2, 0, 0), (2, 16, 2), (1, 32, 4), (4, 8, 2), (4, 32, 2), (5, 8, 2),
                       (5, 16, 4)]:
        M.set_filter_kernel(kind, g, v)
        Y = empty_like_np((A.n, p), A.is_complex)
        B.filter_apply_defect(ctx, M, coef, l1, l2, dev(V), dev(AV), dev(lam), Y)
        outs.append(host(Y))
    M.close()
    ref = clenshaw_apply(As, coef, l1, l2, V)
    R = AV - V * lam
    assert np.max(np.abs(outs[0] - ref)) <= clenshaw_tol(coef, l1 * R, EPS32) + 1e-12
    for y in outs[1:]:
        assert np.array_equal(outs[0], y)


def test_solve_is_the_same_with_every_pinned_kernel(B, ctx):
    """A whole defect-corrected solve on a matrix with a permuted copy: the
    same eigenvalues, bit for bit, whichever kernel runs the filter."""
    A = matrices.anderson(17, 3, 3.5, 5, False)
    lam = np.linalg.eigvalsh(A.to_dense())
    i, c = 2400, 12
    a, b = 0.5 * (lam[i - 1] + lam[i]), 0.5 * (lam[i + c - 1] + lam[i + c])
    M = B.Matrix.from_csr(ctx, A.n, A.rowptr, A.colidx, A.vals)
    got = []
    for kind in (0, 1, 2, 3, 4, 5):
        M.set_filter_kernel(kind)
        r = B.solve(ctx, M, B.default_params(a=a, b=b, p=24, seed=3, filter_precision=B.APF_FILTER_F32_DEFECT))
        got.append(r.eigvals())
        r.close()
    M.close()
    assert np.max(np.abs(got[0] - lam[i:i + c])) <= 1e-10 * np.abs(lam).max()
    for g in got[1:]:
        assert np.array_equal(got[0], g)


def test_set_filter_kernel_rejects_bad_kind(B, ctx):
    A = matrices.anderson(5, 3, 4.0, 3, False)
    M = B.Matrix.from_csr(ctx, A.n, A.rowptr, A.colidx, A.vals)
    for kind in (-1, 6):
        with pytest.raises(B.ApfError) as ei:
            M.set_filter_kernel(kind)
        assert ei.value.status == B.APF_ERR_ARG
    M.close()


@pytest.mark.parametrize("is_complex", [False, True])
def test_column_tiles_on_wide_blocks(B, ctx, is_complex):
    """Blocks wider than one thread group covers (1100 real / 700 complex
    columns): the column-tiled SELL kernel in every tile width against the CSR
    kernel (column slabs) bit for bit, and against the oracle."""
    A = matrices.anderson(12, 3, 3.0, 8, is_complex)
    As = A.to_scipy()
    p = 700 if is_complex else 1100
    lmin, lmax = fsi.gershgorin(As)
    l1, l2 = cb.linear_map(lmin, lmax)
    coef = cb.filter_coefficients(-0.3, 0.1, 33)
    X = rng.uniform_block(13, rng.STREAM_TEST, A.n, p, is_complex)
    ref = clenshaw_apply(As, coef, l1, l2, X)
    M = B.Matrix.from_csr(ctx, A.n, A.rowptr, A.colidx, A.vals)
    outs = []
    for kind, g, v in [(3, 0, 0)] + [(k, g, v) for k in (4, 5) for g, v in CT_SHAPES]:
        M.set_filter_kernel(kind, g, v)
        Y = empty_like_np((A.n, p), is_complex)
        B.filter_apply(ctx, M, coef, l1, l2, dev(X), Y, B.APF_FILTER_F32)
        outs.append(host(Y))
    M.close()
    assert np.max(np.abs(outs[0] - ref)) <= clenshaw_tol(coef, X, EPS32)
    for y in outs[1:]:
        assert np.array_equal(outs[0], y)
