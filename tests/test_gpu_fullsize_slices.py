"""The spectrum-slice workload at full size (48^3 real Anderson, n = 110,592,
eight contiguous slices around E = 0, subspace sizes estimated): properties
that hold at any size, checked on the host in FP64.

 - every slice converges; its pairs lie inside it and their count is what the
   oracle's count estimate predicted for it (stored with the workload) to
   within the estimate's statistical error;
 - every returned pair has ||A v - lambda v|| <= 1e-10 ||A||_est, recomputed
   here with scipy in FP64, and the vectors are orthonormal within a slice
   and obey the Davis-Kahan bound across slices;
 - the slice that a single solve of the same interval would produce has the
   same eigenvalues.
"""
import json
import os

import numpy as np
import pytest

from synth import workloads

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "slices_anderson3d_r_48.json")


@pytest.fixture(scope="module")
def B(gpu_lib):
    from paper_2604_00914_gb300 import binding
    return binding


def test_slice_workload_properties(B):
    w = workloads.anderson3d_r_48_slices()
    A = w.matrix()
    with open(GOLDEN) as f:
        est = json.load(f)["count_estimates"]
    ctx = B.Context(0)
    M = B.Matrix.from_csr(ctx, A.n, A.rowptr, A.colidx, A.vals)
    r = B.solve_slices(ctx, M, w.a, w.b, w.p, B.default_params(seed=w.seed,
                                                              filter_precision=B.APF_FILTER_F32_DEFECT))
    lam, V, st, counts = r.eigvals(), r.eigvecs(A.n, False), r.stats(), r.slice_counts(len(w.a))
    r.close()
    assert r.status == 0
    assert counts.sum() == lam.size and np.all(np.diff(lam) >= 0)
    off = 0
    for s in range(len(w.a)):
        ls = lam[off:off + counts[s]]
        assert np.all((ls >= w.a[s]) & (ls <= w.b[s]))
        # Hutchinson with 16 probes: standard deviation about sqrt(2 e / 16)
        assert abs(counts[s] - est[s]) <= 6.0 * np.sqrt(2.0 * est[s] / 16.0) + 1.0, (s, counts[s], est[s])
        off += counts[s]
    res = np.linalg.norm(A.to_scipy() @ V - V * lam, axis=0)
    assert res.max() <= 1e-10 * st["norm_a"]  # norm_a <= ||A||: conservative
    G = np.abs(V.T @ V - np.eye(lam.size))
    sl = np.repeat(np.arange(len(w.a)), counts)
    same = sl[:, None] == sl[None, :]
    assert G[same].max() < 1e-10
    gap = np.abs(lam[:, None] - lam[None, :]) + np.eye(lam.size)
    bound = (res[:, None] + res[None, :]) / gap
    assert np.all(G[~same] <= 1.01 * bound[~same] + 1e-14)
    # one slice on its own
    s = 3
    one = B.solve(ctx, M, B.default_params(a=w.a[s], b=w.b[s], p=0, seed=w.seed,
                                           filter_precision=B.APF_FILTER_F32_DEFECT))
    lam1 = one.eigvals()
    one.close()
    o = int(counts[:s].sum())
    assert lam1.size == counts[s]
    assert np.max(np.abs(lam1 - lam[o:o + counts[s]])) <= 1e-10 * st["norm_a"]
    M.close()
    ctx.close()
