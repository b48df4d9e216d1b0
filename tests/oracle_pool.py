"""Run the oracle's Alg. 2 (oracle.filter.clenshaw_apply) on column slices of
a block in separate processes (spawned, never forked: the parent may hold a
CUDA context).  The filter acts on each column independently and scipy's
sparse product sums every column in the same order whatever the block width,
so the slices together equal one call on the whole block bit for bit; this
only spreads the work of the full-size comparisons over the host cores.

The matrix and both blocks travel through shared memory."""
from __future__ import annotations

import multiprocessing as mp
import os
from multiprocessing import shared_memory

import numpy as np


def _attach(name, shape, dtype):
    shm = shared_memory.SharedMemory(name=name)
    return shm, np.ndarray(shape, dtype=dtype, buffer=shm.buf)


def _worker(job):
    import scipy.sparse as sp
    from oracle.filter import clenshaw_apply
    (n, nnz, rp, ci, va, vdt, xin, xout, p, bdt, c0, c1, coef, l1, l2) = job
    s1, rowptr = _attach(rp, (n + 1,), np.int64)
    s2, colidx = _attach(ci, (nnz,), np.int32)
    s3, vals = _attach(va, (nnz,), vdt)
    s4, X = _attach(xin, (n, p), bdt)
    s5, Y = _attach(xout, (n, p), bdt)
    A = sp.csr_matrix((vals, colidx.astype(np.int64), rowptr), shape=(n, n))
    Y[:, c0:c1] = clenshaw_apply(A, np.asarray(coef), l1, l2, np.array(X[:, c0:c1]))
    del A, rowptr, colidx, vals, X, Y
    for s in (s1, s2, s3, s4, s5):
        s.close()
    return c1 - c0


def _share(arr):
    shm = shared_memory.SharedMemory(create=True, size=max(arr.nbytes, 1))
    view = np.ndarray(arr.shape, dtype=arr.dtype, buffer=shm.buf)
    view[...] = arr
    return shm


def clenshaw_apply_parallel(A, coef, l1, l2, X, workers=None):
    """oracle.filter.clenshaw_apply(A.to_scipy(), coef, l1, l2, X) with the
    columns dealt to `workers` spawned processes.  A: synth.matrices.CSR."""
    n, p = X.shape
    workers = max(1, min(workers or os.cpu_count() or 1, p))
    shms = [_share(np.ascontiguousarray(A.rowptr, dtype=np.int64)),
            _share(np.ascontiguousarray(A.colidx, dtype=np.int32)),
            _share(np.ascontiguousarray(A.vals)),
            _share(np.ascontiguousarray(X))]
    out = shared_memory.SharedMemory(create=True, size=X.nbytes)
    shms.append(out)
    try:
        edges = np.linspace(0, p, workers + 1).astype(int)
        jobs = [(n, A.nnz, shms[0].name, shms[1].name, shms[2].name, A.vals.dtype, shms[3].name, out.name, p,
                 X.dtype, int(edges[i]), int(edges[i + 1]), list(map(float, coef)), float(l1), float(l2))
                for i in range(workers) if edges[i + 1] > edges[i]]
        with mp.get_context("spawn").Pool(len(jobs)) as pool:
            done = sum(pool.map(_worker, jobs))
        assert done == p
        return np.array(np.ndarray((n, p), dtype=X.dtype, buffer=out.buf))
    finally:
        for s in shms:
            s.close()
            s.unlink()
