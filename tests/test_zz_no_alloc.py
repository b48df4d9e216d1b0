"""apf_gram_noalloc: the Gram product for callers that cannot allocate device
memory (work inside a CUDA graph capture, allocator callbacks, fixed memory
budgets).  It must return what apf_gram returns, call after call, although
every call reuses the same fixed device array for its partial sums.

This file is collected last so that a run stopping at the first failure has
already run every other test; it also passes when run alone.
"""
import numpy as np
import pytest

from gpu_util import EPS64, dev, empty_like_np, host
from synth import rng

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B(gpu_lib):
    from paper_2604_00914_gb300 import binding
    return binding


def _noalloc(B, X, Y, G):
    import torch
    n, pa = X.shape
    pb = Y.shape[1]
    dt = B.APF_C128 if X.is_complex() else B.APF_R64
    stream = torch.cuda.current_stream().cuda_stream
    st = B.Library.load().apf_gram_noalloc(dt, n, pa, pb, X.data_ptr(), X.stride(0), Y.data_ptr(),
                                           Y.stride(0), G.data_ptr(), G.stride(0), stream)
    torch.cuda.synchronize()
    return st


@pytest.mark.parametrize("is_complex", [False, True])
def test_noalloc_gram_matches_gram_twice(B, is_complex):
    """Two calls in a row (different shapes, so different split counts over the
    shared array) both match apf_gram within the Gram test's tolerance."""
    ctx = B.Context(0)
    try:
        for call, (n, pa, pb) in enumerate([(5003, 37, 45), (20000, 160, 160)]):
            X = dev(rng.uniform_block(30 + call, rng.STREAM_TEST, n, pa, is_complex))
            Y = dev(rng.uniform_block(40 + call, rng.STREAM_TEST, n, pb, is_complex))
            G_ref = empty_like_np((pa, pb), is_complex)
            B.gram(ctx, X, Y, G_ref)
            G = empty_like_np((pa, pb), is_complex)
            G.fill_(float("nan"))
            assert _noalloc(B, X, Y, G) == B.APF_OK
            tol = 4 * n * EPS64
            assert np.max(np.abs(host(G) - host(G_ref))) <= tol
            ref = host(X).conj().T @ host(Y)
            assert np.max(np.abs(host(G) - ref)) <= tol
    finally:
        ctx.close()


def test_noalloc_gram_rejects_sizes_beyond_its_array(B):
    """pa * pb elements must fit the 8 MiB array: 1100 x 1100 doubles do not."""
    import torch
    n = 64
    X = torch.zeros((n, 1100), dtype=torch.float64, device="cuda")
    G = torch.zeros((1100, 1100), dtype=torch.float64, device="cuda")
    assert _noalloc(B, X, X, G) == B.APF_ERR_ARG
