"""Every device-side wait ends: a wait that nothing satisfies gives up after
the context's time limit, the call reports APF_ERR_TIMEOUT, and the same
context then solves normally.  The waits are the two-step filter pass's
dependency wait (Alg. 2, two Clenshaw steps per pass) and the small
eigensolver's grid barrier (the Rayleigh-Ritz step of Alg. 4).  Nothing here
faults the GPU: the kernels return by themselves once the limit is reached."""
import time

import numpy as np
import pytest

from synth import matrices

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B(gpu_lib):
    from paper_2604_00914_gb300 import binding
    return binding


def _solve_ok(B, ctx, M, A):
    lam = np.linalg.eigvalsh(A.to_dense())
    i0 = int(np.searchsorted(lam, 0.3))
    a, b = 0.5 * (lam[i0 - 4] + lam[i0 - 3]), 0.5 * (lam[i0 + 2] + lam[i0 + 3])
    r = B.solve(ctx, M, B.default_params(a=a, b=b, p=14, seed=3, filter_precision=B.APF_FILTER_F32_DEFECT))
    got = r.eigvals()
    r.close()
    ref = lam[(lam >= a) & (lam <= b)]
    assert got.size == ref.size and np.max(np.abs(got - ref)) < 1e-9


@pytest.mark.parametrize("which", [0, 1])
def test_unsatisfiable_wait_times_out_and_context_survives(B, which):
    A = matrices.anderson(9, 3, 4.0, 21, True)
    ctx = B.Context(0)
    try:
        M = B.Matrix.from_csr(ctx, A.n, A.rowptr, A.colidx, A.vals)
        ctx.set_wait_limit(1_000_000)  # 1 ms
        t0 = time.perf_counter()
        st = ctx.wait_probe(which, M)
        dt = time.perf_counter() - t0
        assert st == B.APF_ERR_TIMEOUT
        assert dt < 5.0
        ctx.set_wait_limit(0)  # defaults again
        _solve_ok(B, ctx, M, A)
        M.close()
    finally:
        ctx.close()


def test_wait_limit_rejects_bad_values(B):
    ctx = B.Context(0)
    try:
        with pytest.raises(B.ApfError):
            ctx.set_wait_limit(-1)
        with pytest.raises(B.ApfError):
            ctx.set_wait_limit(61_000_000_000)
        assert ctx.wait_probe(7) == B.APF_ERR_ARG
        assert ctx.wait_probe(0, None) == B.APF_ERR_ARG
    finally:
        ctx.close()
