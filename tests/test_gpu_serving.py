"""The serving loop (apf_server_*): independent requests served with
continuous batching on one GPU, admitted by device-memory budget between outer
iterations; the Clenshaw steps of all running FP32-filter requests share one
launch per step.  Each result must equal the result of the same request
solved alone with apf_solve, bit for bit, and match the definition (dense
eigh)."""
import numpy as np
import pytest

from synth import matrices

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B(gpu_lib):
    from paper_2604_00914_gb300 import binding
    return binding


def _gap_interval(lam, i, c):
    return 0.5 * (lam[i - 1] + lam[i]), 0.5 * (lam[i + c - 1] + lam[i + c])


def _requests(B):
    """Real and complex, 2D and 3D, given and estimated p, two filter precisions."""
    out = []
    specs = [
        (matrices.anderson(10, 3, 5.0, 41, False), 300, 12, 24, "F32_DEFECT"),
        (matrices.anderson(10, 3, 4.0, 42, True), 520, 9, 0, "F32_DEFECT"),
        (matrices.laplacian2d_dirichlet(40, 43), 700, 10, 20, "F32_DEFECT"),
        (matrices.ks_like_3d(12, 44, n_wells=6), 80, 8, 16, "F64"),
        (matrices.anderson(9, 3, 6.0, 45, True), 200, 6, 14, "F32"),
    ]
    for A, i, c, p, prec in specs:
        lam = np.linalg.eigvalsh(A.to_dense())
        a, b = _gap_interval(lam, i, c)
        prm = dict(a=a, b=b, p=p, seed=9, filter_precision=getattr(B, "APF_FILTER_" + prec))
        out.append((A, prm, lam[i:i + c]))
    return out


def _alone(B, reqs):
    ctx = B.Context(0)
    res = []
    for A, prm, _ in reqs:
        M = B.Matrix.from_csr(ctx, A.n, A.rowptr, A.colidx, A.vals)
        r = B.solve(ctx, M, B.default_params(**prm), allow_no_convergence=True)
        res.append((r.eigvals(), r.residuals(), r.stats()["iterations"]))
        r.close()
        M.close()
    ctx.close()
    return res


def _served(B, reqs, **kw):
    srv = B.Server(0, **kw)
    tickets = [srv.submit(A.n, A.rowptr, A.colidx, A.vals, B.default_params(**prm)) for A, prm, _ in reqs]
    res, infos = [], []
    for t in tickets:
        r, info = srv.wait(t, allow_no_convergence=True)
        res.append((r.eigvals(), r.residuals(), r.stats()["iterations"]))
        infos.append(info)
        r.close()
    state = srv.state()
    srv.close()
    return res, infos, state


def test_mix_equals_alone_and_definition(B):
    reqs = _requests(B)
    alone = _alone(B, reqs)
    mixed, infos, state = _served(B, reqs, max_concurrent=4)
    assert state["completed"] == len(reqs) and state["peak_running"] >= 2
    # the FP32 requests' steps went out together (real and complex launches)
    assert state["batched_launches"] > 0 and state["widest_batch"] >= 2
    for (A, prm, lam_ref), (la, ra, ia), (lm, rm, im), info in zip(reqs, alone, mixed, infos):
        if prm["filter_precision"] == B.APF_FILTER_F32:  # plain FP32 stalls: compare, do not require 0
            assert info["status"] in (0, B.APF_ERR_NO_CONVERGENCE)
            assert np.array_equal(la, lm) and ia == im
            continue
        assert info["status"] == 0
        assert np.array_equal(la, lm) and np.array_equal(ra, rm) and ia == im
        assert lm.size == lam_ref.size
        assert np.max(np.abs(lm - lam_ref)) <= 1e-10 * np.abs(lam_ref).max() * 10
        assert 0 <= info["queue_ms"] <= info["latency_ms"] and 0 < info["run_ms"] <= info["latency_ms"]


def test_budget_admits_one_at_a_time(B):
    """With a budget of the largest footprint no two requests fit together:
    they run one after another, with the same results."""
    reqs = _requests(B)[:3]
    first, infos, _ = _served(B, reqs, max_concurrent=3)
    budget = max(i["footprint_bytes"] for i in infos)
    again, infos2, state = _served(B, reqs, max_concurrent=3, hbm_budget_bytes=budget)
    assert state["peak_running"] == 1 and state["peak_in_flight_bytes"] <= budget
    for (l1, r1, _), (l2, r2, _) in zip(first, again):
        assert np.array_equal(l1, l2) and np.array_equal(r1, r2)


def test_server_rejects_bad_requests(B):
    A = matrices.anderson(6, 3, 4.0, 3, False)
    srv = B.Server(0, max_concurrent=2, hbm_budget_bytes=1 << 20)
    with pytest.raises(B.ApfError) as ei:  # footprint above the budget
        srv.submit(A.n, A.rowptr, A.colidx, A.vals, B.default_params(a=-0.5, b=0.5, p=8))
    assert ei.value.status == B.APF_ERR_OOM
    srv.close()
    srv = B.Server(0, max_concurrent=2)
    V0 = np.zeros((A.n, 8))
    with pytest.raises(B.ApfError) as ei:  # caller buffers are not kept
        srv.submit(A.n, A.rowptr, A.colidx, A.vals, B.default_params(a=-0.5, b=0.5, p=8, init_block=V0.ctypes.data))
    assert ei.value.status == B.APF_ERR_ARG
    with pytest.raises(B.ApfError) as ei:
        srv.wait(12345)
    assert ei.value.status == B.APF_ERR_ARG
    # a failing solve (interval outside the spectrum) reports its status; the server goes on
    t_bad = srv.submit(A.n, A.rowptr, A.colidx, A.vals, B.default_params(a=50.0, b=60.0, p=8))
    lam = np.linalg.eigvalsh(A.to_dense())
    a, b = _gap_interval(lam, 100, 4)
    t_ok = srv.submit(A.n, A.rowptr, A.colidx, A.vals, B.default_params(a=a, b=b, p=10))
    t_unwaited = srv.submit(A.n, A.rowptr, A.colidx, A.vals, B.default_params(a=a, b=b, p=10))
    with pytest.raises(B.ApfError) as ei:
        srv.wait(t_bad)
    assert ei.value.status == B.APF_ERR_ARG
    r, info = srv.wait(t_ok)
    assert info["status"] == 0 and r.eigvals().size == 4
    with pytest.raises(B.ApfError):  # a ticket is waited for once
        srv.wait(t_ok)
    srv.close()  # frees the result of t_unwaited
    assert np.allclose(r.eigvals(), lam[100:104], atol=1e-9)  # still valid after the server
    r.close()
    assert t_unwaited > t_ok


def test_late_arrivals_join_the_running_batch(B):
    """Continuous batching: requests submitted while another is on the GPU are
    admitted at its next outer iteration, share its filter launches, and
    finish first when they are cheaper; every result equals apf_solve's."""
    import time
    big = matrices.anderson(24, 3, 4.0, 51, True)
    lam_big = np.linalg.eigvalsh(big.to_dense())
    a, b = _gap_interval(lam_big, 7000, 14)
    big_prm = dict(a=a, b=b, p=28, seed=5, filter_precision=B.APF_FILTER_F32_DEFECT)
    small = []
    for k, A in enumerate([matrices.anderson(9, 3, 5.0, 52, False), matrices.laplacian2d_dirichlet(30, 53)]):
        lam = np.linalg.eigvalsh(A.to_dense())
        a, b = _gap_interval(lam, 300, 6)
        small.append((A, dict(a=a, b=b, p=12, seed=6 + k, filter_precision=B.APF_FILTER_F32_DEFECT)))
    reqs = [(big, big_prm, None)] + [(A, prm, None) for A, prm in small]
    alone = _alone(B, reqs)
    srv = B.Server(0, max_concurrent=4)
    t_big = srv.submit(big.n, big.rowptr, big.colidx, big.vals, B.default_params(**big_prm))
    t0 = time.time()
    while srv.state()["running"] < 1 and time.time() - t0 < 30:
        time.sleep(0.005)
    time.sleep(0.05)  # the big request is past its set-up and iterating
    ts = [srv.submit(A.n, A.rowptr, A.colidx, A.vals, B.default_params(**prm)) for A, prm in small]
    got = []
    for t in [t_big] + ts:
        r, info = srv.wait(t)
        got.append((r.eigvals(), r.residuals(), r.stats()["iterations"], info))
        r.close()
    state = srv.state()
    srv.close()
    assert state["peak_running"] >= 2 and state["widest_batch"] >= 2
    for (la, ra, ia), (lm, rm, im, info) in zip(alone, got):
        assert info["status"] == 0
        assert np.array_equal(la, lm) and np.array_equal(ra, rm) and ia == im
