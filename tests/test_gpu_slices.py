"""Spectrum slicing through apf_solve_slices (Sec. 1: the spectrum is cut into
slices whose eigenpairs are computed independently).

Every slice must give what the definition gives for its interval (dense eigh),
and what a single solve of that interval gives, while one filter launch per
Clenshaw step serves all slices.
"""
import numpy as np
import pytest

from synth import matrices

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


def _gap_interval(lam, lo_idx, cnt):
    """[a, b] holding lam[lo_idx : lo_idx + cnt], ends in the middle of the gaps."""
    return 0.5 * (lam[lo_idx - 1] + lam[lo_idx]), 0.5 * (lam[lo_idx + cnt - 1] + lam[lo_idx + cnt])


def _slices(lam, specs):
    a, b = zip(*[_gap_interval(lam, i, c) for i, c in specs])
    return np.array(a), np.array(b)


def _run_slices(B, ctx, A, a, b, p, seed, kernel=0, **kw):
    M = B.Matrix.from_csr(ctx, A.n, A.rowptr, A.colidx, A.vals)
    if kernel:
        M.set_filter_kernel(kernel)
    prm = B.default_params(seed=seed, **kw)
    r = B.solve_slices(ctx, M, a, b, p, prm, allow_no_convergence=True)
    out = dict(status=r.status, lam=r.eigvals(), V=r.eigvecs(A.n, A.is_complex), res=r.residuals(),
               stats=r.stats(), hist=r.history(), counts=r.slice_counts(len(a)))
    r.close()
    M.close()
    return out


def _run_single(B, ctx, A, a, b, p, seed, **kw):
    M = B.Matrix.from_csr(ctx, A.n, A.rowptr, A.colidx, A.vals)
    r = B.solve(ctx, M, B.default_params(a=a, b=b, p=p, seed=seed, **kw), allow_no_convergence=True)
    out = dict(status=r.status, lam=r.eigvals(), stats=r.stats())
    r.close()
    M.close()
    return out


def _check_against_definition(out, A, lam, a, b, tol=1e-10):
    normA = np.abs(lam).max()
    norm_est = out["stats"]["norm_a"]
    assert out["status"] == 0
    # per-slice counts (input order) and the union, ascending
    ref_counts = [int(np.sum((lam >= lo) & (lam <= hi))) for lo, hi in zip(a, b)]
    assert list(out["counts"]) == ref_counts
    inside = np.zeros(lam.size, bool)
    for lo, hi in zip(a, b):
        inside |= (lam >= lo) & (lam <= hi)
    lam_ref = lam[inside]
    assert out["lam"].size == lam_ref.size
    assert np.all(np.diff(out["lam"]) >= 0)
    assert np.max(np.abs(out["lam"] - lam_ref)) <= tol * normA
    V = out["V"]
    R = A.to_scipy() @ V - V * out["lam"]
    res = np.linalg.norm(R, axis=0)
    assert norm_est <= normA * (1 + 1e-12)
    assert res.max() <= tol * normA
    assert np.max(np.abs(out["res"] - res / norm_est)) < 1e-12
    # within a slice the vectors come out of one Rayleigh-Ritz basis; across
    # slices |v_i^H v_j| <= (||r_i|| + ||r_j||) / |lam_i - lam_j| (Davis-Kahan)
    G = np.abs(V.conj().T @ V - np.eye(V.shape[1]))
    sl = np.searchsorted(np.sort(np.concatenate([a, b])), out["lam"]) // 2
    for i in range(G.shape[0]):
        for j in range(G.shape[1]):
            if i == j or sl[i] == sl[j]:
                assert G[i, j] < 1e-10
            else:
                bound = (res[i] + res[j]) / abs(out["lam"][i] - out["lam"][j])
                assert G[i, j] <= 1.01 * bound + 1e-14


@pytest.mark.parametrize("prec", PREC)
@pytest.mark.parametrize("is_complex", [False, True])
def test_slices_match_definition(B, ctx, prec, is_complex):
    """Four disjoint slices of different widths (so different degrees), given
    out of order, of a 3D Anderson matrix; counts 5, 9, 3 and 12."""
    A = matrices.anderson(10, 3, 5.0, 21, is_complex)
    lam = np.linalg.eigvalsh(A.to_dense())
    a, b = _slices(lam, [(520, 9), (300, 5), (700, 3), (90, 12)])
    p = np.array([16, 12, 8, 20])
    out = _run_slices(B, ctx, A, a, b, p, 5, filter_precision=getattr(B, "APF_FILTER_" + prec))
    _check_against_definition(out, A, lam, a, b)


@pytest.mark.slow
def test_wide_slices_beyond_1024_columns(B, ctx):
    """Twelve slices whose subspaces add up to more than 1024 columns (the
    batched filter then runs in column tiles): every slice as the definition
    gives it.  Real 3D Anderson model, 16^3."""
    A = matrices.anderson(16, 3, 5.0, 23, False)
    lam = np.linalg.eigvalsh(A.to_dense())
    specs = [(200 + 160 * s, 60 + 5 * (s % 3)) for s in range(12)]
    a, b = _slices(lam, specs)
    p = np.array([c + 36 for _, c in specs])
    assert p.sum() > 1024
    out = _run_slices(B, ctx, A, a, b, p, 5, filter_precision=B.APF_FILTER_F32_DEFECT)
    assert out["stats"]["p_used"] == p.sum()
    ref_counts = [int(np.sum((lam >= lo) & (lam <= hi))) for lo, hi in zip(a, b)]
    assert list(out["counts"]) == ref_counts
    inside = np.zeros(lam.size, bool)
    for lo, hi in zip(a, b):
        inside |= (lam >= lo) & (lam <= hi)
    assert np.max(np.abs(out["lam"] - lam[inside])) <= 1e-10 * np.abs(lam).max()
    res = np.linalg.norm(A.to_scipy() @ out["V"] - out["V"] * out["lam"], axis=0)
    assert res.max() <= 1e-10 * np.abs(lam).max()


@pytest.mark.parametrize("prec", PREC)
def test_slice_graph_replay_gives_the_same_solve(B, ctx, prec):
    """Recurring batched filter applications (the same per-column degrees and
    widths: a fixed degree, before the first lock) replay as one CUDA graph
    for all slices: the same eigenvalues, residuals, counts and launch
    counters as plain launches.  The FP32 step is pinned to one step per
    launch: the two-step kernel's pass counters rule out graphs."""
    A = matrices.anderson(10, 3, 5.0, 21, False)
    lam = np.linalg.eigvalsh(A.to_dense())
    a, b = _slices(lam, [(520, 9), (300, 5), (90, 12)])
    p = np.array([16, 12, 20])
    kw = dict(filter_precision=getattr(B, "APF_FILTER_" + prec), k_fixed=300, kernel=1)
    on = _run_slices(B, ctx, A, a, b, p, 5, filter_graphs=1, **kw)
    off = _run_slices(B, ctx, A, a, b, p, 5, filter_graphs=0, **kw)
    assert on["status"] == off["status"] == 0
    assert np.array_equal(on["lam"], off["lam"]) and np.array_equal(on["res"], off["res"])
    assert list(on["counts"]) == list(off["counts"])
    for key in ("iterations", "filter_launches", "filter_steps", "spmv_columns", "gpu_launches"):
        assert on["stats"][key] == off["stats"][key], key
    assert on["stats"]["filter_graph_replays"] > 0 and off["stats"]["filter_graph_replays"] == 0
    _check_against_definition(on, A, lam, a, b)


@pytest.mark.parametrize("prec", PREC)
def test_slices_equal_single_solves(B, ctx, prec):
    """Each slice finds the eigenvalues a single solve of its interval finds,
    and the batched run needs fewer filter launches than the single runs."""
    A = matrices.anderson(9, 3, 4.0, 8, True)
    lam = np.linalg.eigvalsh(A.to_dense())
    a, b = _slices(lam, [(100, 6), (360, 10), (600, 4)])
    p = np.array([12, 16, 10])
    kw = dict(filter_precision=getattr(B, "APF_FILTER_" + prec))
    out = _run_slices(B, ctx, A, a, b, p, 3, **kw)
    assert out["status"] == 0
    launches = 0
    got = []
    for s in range(3):
        one = _run_single(B, ctx, A, a[s], b[s], int(p[s]), 3, **kw)
        assert one["status"] == 0
        got.append(one["lam"])
        launches += one["stats"]["filter_launches"]
        assert out["counts"][s] == one["lam"].size
    ref = np.concatenate(got)
    assert np.max(np.abs(np.sort(ref) - out["lam"])) <= 1e-10 * np.abs(lam).max()
    assert out["stats"]["filter_launches"] < launches
    # one pass of the recurrence per iteration, as long as the highest degree
    assert out["stats"]["filter_steps"] <= sum(int(h["degree"]) for h in out["hist"])


def test_one_slice_is_a_single_solve(B, ctx):
    """With one slice the batched filter does the single solve's arithmetic
    (same start block, same coefficients): the results are identical."""
    A = matrices.anderson(9, 3, 4.0, 12, False)
    lam = np.linalg.eigvalsh(A.to_dense())
    a, b = _slices(lam, [(400, 7)])
    out = _run_slices(B, ctx, A, a, b, np.array([14]), 6)
    one = _run_single(B, ctx, A, a[0], b[0], 14, 6)
    assert out["status"] == 0 and one["status"] == 0
    assert np.array_equal(out["lam"], one["lam"])
    assert out["stats"]["iterations"] == one["stats"]["iterations"]


def test_slices_reject_bad_input(B, ctx):
    A = matrices.anderson(6, 3, 4.0, 3, False)
    M = B.Matrix.from_csr(ctx, A.n, A.rowptr, A.colidx, A.vals)
    prm = B.default_params()
    bad = [
        ([-1.0, -0.5], [0.0, 0.5], [4, 4]),      # overlapping
        ([0.0, -1.0], [0.5, 0.2], [4, 4]),       # overlapping, out of order
        ([-1.0], [-2.0], [4]),                   # a > b
        ([-1.0, 1.0], [-0.5, 1.5], [4, -1]),     # p < 0 (0 asks for an estimate)
        ([-1.0, 1.0], [-0.5, 1.5], [200, 100]),  # sum(p) > n
    ]
    for a, b, p in bad:
        with pytest.raises(B.ApfError) as ei:
            B.solve_slices(ctx, M, a, b, p, prm)
        assert ei.value.status == B.APF_ERR_ARG
    V0 = np.zeros((A.n, 4))
    with pytest.raises(B.ApfError) as ei:
        B.solve_slices(ctx, M, [-1.0], [-0.5], [4], B.default_params(init_block=V0.ctypes.data, init_on_device=0))
    assert ei.value.status == B.APF_ERR_ARG
    # slice counts only for a result of apf_solve_slices, with its slice count
    lam = np.linalg.eigvalsh(A.to_dense())
    a, b = _slices(lam, [(100, 3), (150, 2)])
    r = B.solve_slices(ctx, M, a, b, [8, 8], prm)
    with pytest.raises(B.ApfError):
        r.slice_counts(3)
    assert list(r.slice_counts(2)) == [3, 2]
    r.close()
    r1 = B.solve(ctx, M, B.default_params(a=a[0], b=b[0], p=8))
    with pytest.raises(B.ApfError):
        r1.slice_counts(1)
    r1.close()
    M.close()
