"""The eigenvalue-count estimate and the estimated subspace size (Sec. 3.4)
on the GPU, against oracle/trace.py on the same seeded +-1 probes."""
import numpy as np
import pytest

from gpu_util import EPS32, EPS64, clenshaw_tol
from oracle import chebyshev as cb
from oracle import trace
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


def _gap_interval(lam, i, c):
    return 0.5 * (lam[i - 1] + lam[i]), 0.5 * (lam[i + c - 1] + lam[i + c])


@pytest.mark.parametrize("prec", ["F64", "F32"])
@pytest.mark.parametrize("is_complex", [False, True])
@pytest.mark.parametrize("m", [1, 24, 200])
def test_count_estimate_matches_oracle(B, ctx, prec, is_complex, m):
    """Widths 1, 24 and 200 probes (200: several column tiles and a ragged tail)."""
    A = matrices.anderson(10, 3, 5.0, 31, is_complex)
    lam = np.linalg.eigvalsh(A.to_dense())
    a, b = _gap_interval(lam, 400, 15)
    l1, l2 = cb.linear_map(lam[0] - 0.2, lam[-1] + 0.2)
    coef = cb.filter_coefficients(l1 * a + l2, l1 * b + l2, 300, cb.DAMP_LANCZOS_M, 0.5)
    M = B.Matrix.from_csr(ctx, A.n, A.rowptr, A.colidx, A.vals)
    got = B.count_estimate(ctx, M, coef, l1, l2, m, 77, precision=getattr(B, "APF_FILTER_" + prec))
    M.close()
    Z = rng.rademacher_block(77, rng.STREAM_TRACE, A.n, m)
    ref = trace.trace_estimate(A.to_scipy(), coef, l1, l2, Z)
    # each of the n terms of a probe's sum carries at most the Alg. 2 entry bound
    tol = A.n * clenshaw_tol(coef, Z, EPS64 if prec == "F64" else EPS32)
    assert abs(got - ref) <= tol, (got, ref, tol)


def _expected_p(B, A, st, a, b, m, seed, prec_eps, mu=1.8):
    """p from the oracle's estimate with the bounds the solve used and the
    interval's maximum degree k = ceil(2.5 k^(1)) (Eq. (compute_k_1))."""
    l1, l2 = cb.linear_map(st["lambda_min"], st["lambda_max"])
    am, bm = l1 * a + l2, l1 * b + l2
    k = cb.maximum_degree(cb.initial_degree(am, bm, 1.4), 2.5)
    coef = cb.filter_coefficients(am, bm, k, cb.DAMP_LANCZOS_M, 0.5)
    Z = rng.rademacher_block(seed, rng.STREAM_TRACE, A.n, m)
    e = trace.trace_estimate(A.to_scipy(), coef, l1, l2, Z)
    # sizes the rule gives for any estimate within `d` of the oracle's
    d = 1e-9 if prec_eps == EPS64 else 1e-3
    lo, hi = trace.subspace_size(e - d, mu, A.n, 1024), trace.subspace_size(e + d, mu, A.n, 1024)
    return e, d, set(range(lo, hi + 1))


@pytest.mark.parametrize("prec", ["F64", "F32_DEFECT"])
def test_solve_with_estimated_subspace_size(B, ctx, prec):
    A = matrices.anderson(10, 3, 5.0, 32, True)
    lam = np.linalg.eigvalsh(A.to_dense())
    a, b = _gap_interval(lam, 600, 14)
    M = B.Matrix.from_csr(ctx, A.n, A.rowptr, A.colidx, A.vals)
    prm = B.default_params(a=a, b=b, p=0, seed=11, filter_precision=getattr(B, "APF_FILTER_" + prec))
    r = B.solve(ctx, M, prm)
    st = r.stats()
    lam_got = r.eigvals()
    r.close()
    M.close()
    assert np.max(np.abs(lam_got - lam[600:614])) <= 1e-10 * np.abs(lam).max()
    e, d, ps = _expected_p(B, A, st, a, b, 32, 11, EPS64 if prec == "F64" else EPS32)
    assert st["k_max"] == cb.maximum_degree(st["k1"], 2.5)
    assert abs(st["trace_estimate"] - e) <= d and st["p_used"] in ps
    assert st["p_used"] == trace.subspace_size(st["trace_estimate"], 1.8, A.n, 1024)
    assert st["p_used"] >= 14


def test_slices_with_estimated_sizes(B, ctx):
    """Two of three slices estimate their sizes in one batched filter pass."""
    A = matrices.anderson(9, 3, 4.0, 33, False)
    lam = np.linalg.eigvalsh(A.to_dense())
    iv = [_gap_interval(lam, i, c) for i, c in [(150, 8), (400, 5), (620, 11)]]
    a = np.array([x for x, _ in iv])
    b = np.array([y for _, y in iv])
    M = B.Matrix.from_csr(ctx, A.n, A.rowptr, A.colidx, A.vals)
    r = B.solve_slices(ctx, M, a, b, [0, 10, 0], B.default_params(seed=4))
    st = r.stats()
    counts = r.slice_counts(3)
    r.close()
    M.close()
    assert list(counts) == [8, 5, 11]
    # the stats carry sums over the slices
    e0, d, p0 = _expected_p(B, A, st, a[0], b[0], 32, 4, EPS64)
    e2, d, p2 = _expected_p(B, A, st, a[2], b[2], 32, 4, EPS64)
    assert abs(st["trace_estimate"] - (e0 + e2)) <= 2 * d
    assert st["p_used"] in {10 + x + y for x in p0 for y in p2}


def test_estimate_rejects_bad_arguments(B, ctx):
    A = matrices.anderson(5, 3, 4.0, 3, False)
    M = B.Matrix.from_csr(ctx, A.n, A.rowptr, A.colidx, A.vals)
    coef = np.ones(5)
    for m, prec in [(0, B.APF_FILTER_F64), (10, B.APF_FILTER_F32_DEFECT)]:
        with pytest.raises(B.ApfError) as ei:
            B.count_estimate(ctx, M, coef, 0.1, 0.0, m, 1, precision=prec)
        assert ei.value.status == B.APF_ERR_ARG
    V0 = np.zeros((A.n, 4))
    with pytest.raises(B.ApfError) as ei:  # p = 0 with a caller block
        B.solve(ctx, M, B.default_params(a=-0.5, b=0.5, p=0, init_block=V0.ctypes.data))
    assert ei.value.status == B.APF_ERR_ARG
    with pytest.raises(B.ApfError) as ei:  # p = 0 needs mu > 0
        B.solve(ctx, M, B.default_params(a=-0.5, b=0.5, p=0, mu=0.0))
    assert ei.value.status == B.APF_ERR_ARG
    M.close()
