"""GPU parity of whole solves (Alg. 4) against the oracle, through the C ABI.

The bar: the same eigenvalue count in [a, b] as the definition (dense eigh)
and as the oracle's AdaPolySI, eigenvalues within 1e-10 ||A||, residuals
||A v - lambda v|| / ||A|| <= 1e-10 recomputed here on the host in FP64, and
orthonormal eigenvectors.  ||A|| is the spectral radius (max |lambda|).
"""
import numpy as np
import pytest
import scipy.sparse as sp

from oracle import chebyshev as cb
from oracle import dense, fsi
from synth import matrices, rng, workloads

pytestmark = pytest.mark.gpu

PREC = ["F64", "F32_DEFECT"]


@pytest.fixture(scope="module")
def B(gpu_lib):
    from paper_2604_00914_gb300 import binding
    return binding


@pytest.fixture(scope="module")
def ctx(B):
    c = B.Context(0)
    yield c
    c.close()


def _prec(B, name):
    return getattr(B, "APF_FILTER_" + name)


def _solve(B, ctx, A, a, b, p, seed, kernel=0, **kw):
    M = B.Matrix.from_csr(ctx, A.n, A.rowptr, A.colidx, A.vals)
    if kernel:
        M.set_filter_kernel(kernel)
    prm = B.default_params(a=a, b=b, p=p, seed=seed, **kw)
    r = B.solve(ctx, M, prm, allow_no_convergence=True)
    out = dict(status=r.status, lam=r.eigvals(), V=r.eigvecs(A.n, A.is_complex), res=r.residuals(),
               stats=r.stats(), hist=r.history())
    r.close()
    M.close()
    return out


def _check(out, A, lam_ref, tol=1e-10):
    As = A.to_scipy()
    # ||A|| is the true spectral radius (dense eigh)
    normA = np.abs(np.linalg.eigvalsh(A.to_dense())).max()
    assert out["status"] == 0
    assert out["lam"].size == lam_ref.size, (out["lam"].size, lam_ref.size)
    assert np.max(np.abs(out["lam"] - lam_ref)) <= tol * normA
    V = out["V"]
    # convergence test of Sec. 4, ||r|| <= tau_c ||A||, against the true ||A||:
    # the solver locks against a lower bound of it (Lanczos Ritz values)
    norm_est = out["stats"]["norm_a"]
    assert 0.5 * normA <= norm_est <= normA * (1 + 1e-12)
    res = np.linalg.norm(As @ V - V * out["lam"], axis=0)
    assert res.max() <= tol * normA, res.max() / normA
    assert np.max(np.abs(V.conj().T @ V - np.eye(V.shape[1]))) < 1e-10
    assert np.max(np.abs(out["res"] - res / norm_est)) < 1e-12


def _interval_around(lam, centre, cnt):
    i0 = int(np.searchsorted(lam, centre))
    lo, hi = i0 - cnt // 2, i0 - cnt // 2 + cnt
    return 0.5 * (lam[lo - 1] + lam[lo]), 0.5 * (lam[hi - 1] + lam[hi])


@pytest.mark.parametrize("prec", PREC)
def test_lap2d_workload_matches_definition_and_oracle(B, ctx, prec):
    w = workloads.lap2d_32()
    A = w.matrix()
    lam_ref, _ = dense.interior_eigenpairs(A.to_dense(), w.a, w.b)
    out = _solve(B, ctx, A, w.a, w.b, w.p, w.seed, filter_precision=_prec(B, prec))
    _check(out, A, lam_ref)
    # the oracle's Alg. 4 from the same start block
    V0 = rng.uniform_block(w.seed, rng.STREAM_INIT_BLOCK, A.n, w.p, False)
    v0 = rng.uniform_block(w.seed, rng.STREAM_LANCZOS, A.n, 1, False)[:, 0]
    ro = fsi.adapolysi(A.to_scipy(), w.a, w.b, fsi.Params(p=w.p), V0, v0)
    assert ro.eigvals.size == out["lam"].size
    assert np.max(np.abs(ro.eigvals - out["lam"])) <= 1e-10 * 8.5
    st = out["stats"]
    assert st["k1"] == ro.stats["setup"]["k1"] and st["k_max"] == ro.stats["setup"]["k"]
    if prec == "F64":
        # same arithmetic path as the oracle: the same degree sequence, up to the last iterations
        gd = [int(h["degree"]) for h in out["hist"]]
        od = [h["degree"] for h in ro.stats["history"]]
        assert gd[:3] == od[:3]


@pytest.mark.parametrize("prec", PREC)
def test_complex_anderson_small(B, ctx, prec):
    A = matrices.anderson(10, 3, 4.0, 7, True)
    lam = np.linalg.eigvalsh(A.to_dense())
    a, b = _interval_around(lam, 0.0, 11)
    out = _solve(B, ctx, A, a, b, 20, 7, filter_precision=_prec(B, prec))
    _check(out, A, lam[(lam >= a) & (lam <= b)])
    assert dense.interval_count(A.to_dense(), a, b) == out["lam"].size
    # the statistics name the FP32 step kernel that ran (none for the FP64 filter)
    st = out["stats"]
    if prec == "F64":
        assert st["filter_kind"] == -1
    else:
        assert st["filter_kind"] in (1, 2, 3, 4) and st["filter_g"] in (4, 8, 16, 32) and st["filter_vpt"] >= 1


@pytest.mark.parametrize("prec", PREC)
def test_ks_like_small_low_end(B, ctx, prec):
    """Kohn-Sham-like real case: an interval in the lower part of the spectrum."""
    A = matrices.ks_like_3d(12, 3, n_wells=6)
    lam = np.linalg.eigvalsh(A.to_dense())
    a, b = _interval_around(lam, lam[60], 9)
    out = _solve(B, ctx, A, a, b, 16, 3, filter_precision=_prec(B, prec))
    _check(out, A, lam[(lam >= a) & (lam <= b)])


def test_fixed_jackson_degree(B, ctx):
    A = matrices.anderson(9, 3, 3.0, 2, False)
    lam = np.linalg.eigvalsh(A.to_dense())
    a, b = _interval_around(lam, -1.5, 5)
    out = _solve(B, ctx, A, a, b, 20, 2, k_fixed=250, damping=B.APF_DAMP_JACKSON)
    _check(out, A, lam[(lam >= a) & (lam <= b)])
    assert all(int(h["degree"]) == 250 for h in out["hist"])
    # the oracle converges in the same number of iterations from the same start
    V0 = rng.uniform_block(2, rng.STREAM_INIT_BLOCK, A.n, 20, False)
    v0 = rng.uniform_block(2, rng.STREAM_LANCZOS, A.n, 1, False)[:, 0]
    ro = fsi.adapolysi(A.to_scipy(), a, b, fsi.Params(p=20, k_fixed=250, damping=cb.DAMP_JACKSON), V0, v0)
    assert ro.stats["iterations"] == out["stats"]["iterations"]


def _stall_matrix(seed):
    cs = np.linspace(0.3, 1.0, 100)
    lam = np.sort(np.concatenate([-cs, cs, [-0.05, -0.02, 0.03, 0.06]]))
    n = lam.size
    Q, _ = np.linalg.qr(rng.uniform_block(seed, rng.STREAM_TEST, n, n, False))
    Ad = (Q * lam) @ Q.T
    Ad = 0.5 * (Ad + Ad.T)
    M = sp.csr_matrix(Ad)
    return matrices.CSR(n=n, rowptr=M.indptr.astype(np.int64), colidx=M.indices.astype(np.int32), vals=M.data)


def test_spurious_rule_ends_stall(B, ctx):
    """Sec. 3.3.2 mechanism (see the oracle test of the same name)."""
    A = _stall_matrix(2)
    kw = dict(k_fixed=20, damping=B.APF_DAMP_JACKSON, max_iter=30)
    on = _solve(B, ctx, A, -0.1, 0.1, 15, 2, spurious_rule=1, **kw)
    assert on["status"] == 0 and on["stats"]["iterations"] <= 12
    assert np.allclose(on["lam"], [-0.05, -0.02, 0.03, 0.06], atol=1e-11)
    off = _solve(B, ctx, A, -0.1, 0.1, 15, 2, spurious_rule=0, **kw)
    assert off["status"] == B.APF_ERR_NO_CONVERGENCE and off["stats"]["iterations"] == 30


def test_plain_fp32_filter_stalls_defect_does_not(B, ctx):
    """The plain FP32 recurrence cannot reach 1e-10 (it stalls near single
    precision); the defect form reaches it with the FP64 answer."""
    w = workloads.lap2d_32()
    A = w.matrix()
    f32 = _solve(B, ctx, A, w.a, w.b, w.p, w.seed, filter_precision=B.APF_FILTER_F32, max_iter=25)
    assert f32["status"] == B.APF_ERR_NO_CONVERGENCE
    lam_ref, _ = dense.interior_eigenpairs(A.to_dense(), w.a, w.b)
    dfc = _solve(B, ctx, A, w.a, w.b, w.p, w.seed, filter_precision=B.APF_FILTER_F32_DEFECT)
    _check(dfc, A, lam_ref)


def test_init_block_equals_seeded_generator(B, ctx):
    w = workloads.lap2d_32()
    A = w.matrix()
    V0 = np.ascontiguousarray(rng.uniform_block(w.seed, rng.STREAM_INIT_BLOCK, A.n, w.p, False))
    a = _solve(B, ctx, A, w.a, w.b, w.p, w.seed)
    b = _solve(B, ctx, A, w.a, w.b, w.p, w.seed, init_block=V0.ctypes.data, init_on_device=0)
    assert np.array_equal(a["lam"], b["lam"])


def test_sell_ingest_equals_csr(B, ctx):
    A = matrices.anderson(8, 3, 4.0, 9, True)
    lam = np.linalg.eigvalsh(A.to_dense())
    a, b = _interval_around(lam, 0.3, 7)
    perm, cptr, clen, ci, vals = matrices.csr_to_sell(A, 8, 32)
    M1 = B.Matrix.from_csr(ctx, A.n, A.rowptr, A.colidx, A.vals)
    M2 = B.Matrix.from_sell(ctx, A.n, 8, 32, perm, cptr, clen, ci, vals)
    assert M1.info() == M2.info()
    prm = B.default_params(a=a, b=b, p=14, seed=9)
    r1, r2 = B.solve(ctx, M1, prm), B.solve(ctx, M2, prm)
    assert np.array_equal(r1.eigvals(), r2.eigvals())
    assert r1.eigvals().size == int(np.sum((lam >= a) & (lam <= b)))


def test_rejects_bad_input(B, ctx):
    A = matrices.anderson(5, 3, 4.0, 3, True)
    vals = A.vals.copy()
    vals[1] += 0.5  # breaks A = A^H
    with pytest.raises(B.ApfError) as ei:
        B.Matrix.from_csr(ctx, A.n, A.rowptr, A.colidx, vals)
    assert ei.value.status == B.APF_ERR_NOT_HERMITIAN
    bad = A.colidx.copy()
    bad[0] = A.n + 3
    with pytest.raises(B.ApfError) as ei:
        B.Matrix.from_csr(ctx, A.n, A.rowptr, bad, A.vals)
    assert ei.value.status == B.APF_ERR_ARG
    M = B.Matrix.from_csr(ctx, A.n, A.rowptr, A.colidx, A.vals)
    for kw in (dict(a=1.0, b=0.0, p=4), dict(a=-0.1, b=0.1, p=-1), dict(a=50.0, b=60.0, p=4),
               dict(a=-0.1, b=0.1, p=A.n + 1)):
        with pytest.raises(B.ApfError) as ei:
            B.solve(ctx, M, B.default_params(**kw))
        assert ei.value.status == B.APF_ERR_ARG


def test_matrix_without_stored_diagonal(B, ctx):
    """Rows without a diagonal entry (zero diagonal) are handled by ingest."""
    A = matrices.anderson(9, 3, 0.0, 4, True)
    keep = A.colidx != np.repeat(np.arange(A.n), np.diff(A.rowptr))
    rows = np.repeat(np.arange(A.n), np.diff(A.rowptr))[keep]
    M = sp.csr_matrix((A.vals[keep], (rows, A.colidx[keep])), shape=(A.n, A.n))
    A2 = matrices.CSR(n=A.n, rowptr=M.indptr.astype(np.int64), colidx=M.indices.astype(np.int32), vals=M.data)
    lam = np.linalg.eigvalsh(A2.to_dense())
    a, b = _interval_around(lam, 1.1, 6)
    out = _solve(B, ctx, A2, a, b, 20, 4)
    _check(out, A2, lam[(lam >= a) & (lam <= b)])


@pytest.mark.parametrize("prec", ["F64", "F32", "F32_DEFECT"])
def test_graph_replay_gives_the_same_solve(B, ctx, prec):
    """Recurring filter applications replayed as CUDA graphs do the same work
    as plain launches: identical eigenvalues, residuals and counters."""
    A = matrices.anderson(9, 3, 4.0, 14, True)
    lam = np.linalg.eigvalsh(A.to_dense())
    a, b = _interval_around(lam, 0.4, 8)
    kw = dict(filter_precision=_prec(B, prec), max_iter=12 if prec == "F32" else 50)
    on = _solve(B, ctx, A, a, b, 16, 5, filter_graphs=1, **kw)
    off = _solve(B, ctx, A, a, b, 16, 5, filter_graphs=0, **kw)
    assert on["status"] == off["status"]
    assert np.array_equal(on["lam"], off["lam"]) and np.array_equal(on["res"], off["res"])
    for key in ("iterations", "filter_launches", "filter_steps", "spmv_columns", "gpu_launches"):
        assert on["stats"][key] == off["stats"][key], key
    assert off["stats"]["filter_graph_replays"] == 0
    if prec != "F32":
        assert on["status"] == 0


@pytest.mark.parametrize("prec", ["F64", "F32_DEFECT"])
def test_graph_replay_runs_at_a_fixed_degree(B, ctx, prec):
    """At a fixed degree every outer iteration before the first lock repeats
    the same filter application, so from the third one on it replays as a
    graph; the result equals the plain launches'.  The FP32 step is pinned
    to one step per launch (the two-step kernel is never captured)."""
    A = matrices.anderson(9, 3, 4.0, 14, True)
    lam = np.linalg.eigvalsh(A.to_dense())
    a, b = _interval_around(lam, 0.4, 8)
    kw = dict(filter_precision=_prec(B, prec), k_fixed=300, kernel=1)
    on = _solve(B, ctx, A, a, b, 16, 5, filter_graphs=1, **kw)
    off = _solve(B, ctx, A, a, b, 16, 5, filter_graphs=0, **kw)
    assert on["status"] == off["status"] == 0
    assert np.array_equal(on["lam"], off["lam"]) and np.array_equal(on["res"], off["res"])
    assert on["stats"]["filter_graph_replays"] > 0 and off["stats"]["filter_graph_replays"] == 0
