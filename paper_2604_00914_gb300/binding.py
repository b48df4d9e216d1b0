"""ctypes binding of libapf (include/apf.h): argument marshalling only.

Every computation runs in the CUDA library; this module converts Python
objects (numpy arrays, torch CUDA tensors, ints, floats) into the C ABI's
plain pointers and sizes, and raises ``ApfError`` on a non-zero status.
Loading fails loudly when the in-tree library has not been built.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libapf.so")

APF_OK = 0
APF_ERR_ARG = 1
APF_ERR_OOM = 2
APF_ERR_CUDA = 3
APF_ERR_NOT_HERMITIAN = 4
APF_ERR_CHOL = 5
APF_ERR_NO_CONVERGENCE = 6
APF_ERR_EIGH = 7
APF_ERR_TIMEOUT = 8
APF_ERR_NOT_READY = 9

APF_R64 = 0
APF_C128 = 1

APF_DAMP_LANCZOS_M = 0
APF_DAMP_JACKSON = 1
APF_DAMP_NONE = 2

APF_FILTER_F64 = 0
APF_FILTER_F32 = 1
APF_FILTER_F32_DEFECT = 2

APF_MAX_P = 1024
APF_MAX_SUM_P = 8192

HISTORY_FIELDS = ("degree", "width", "e", "locked", "n_lock", "max_res_in")


class apf_params(C.Structure):
    _fields_ = [
        ("a", C.c_double), ("b", C.c_double), ("p", C.c_int64),
        ("k_fixed", C.c_int32), ("damping", C.c_int32),
        ("C", C.c_double), ("k_ratio", C.c_double), ("m_d", C.c_double),
        ("tau_a", C.c_double), ("tau_c", C.c_double),
        ("max_iter", C.c_int32), ("lanczos_steps", C.c_int32),
        ("bound_pad", C.c_double),
        ("filter_precision", C.c_int32), ("spurious_rule", C.c_int32),
        ("seed", C.c_uint64), ("init_block", C.c_void_p),
        ("init_on_device", C.c_int32), ("max_degree_cap", C.c_int32),
        ("mu", C.c_double), ("trace_probes", C.c_int32), ("filter_graphs", C.c_int32),
        ("gram_tensor_cores", C.c_int32),
    ]


class apf_stats(C.Structure):
    _fields_ = [
        ("iterations", C.c_int32), ("k1", C.c_int32), ("k_max", C.c_int32),
        ("avg_degree", C.c_double), ("spmv_columns", C.c_int64),
        ("filter_launches", C.c_int64), ("gpu_launches", C.c_int64),
        ("lambda_min", C.c_double), ("lambda_max", C.c_double), ("norm_a", C.c_double),
        ("ms_total", C.c_double), ("ms_setup", C.c_double), ("ms_filter", C.c_double),
        ("ms_orth", C.c_double), ("ms_rr", C.c_double), ("ms_check", C.c_double),
        ("filter_kernel_ms", C.c_double), ("filter_bytes", C.c_double),
        ("max_residual", C.c_double),
        ("filter_steps", C.c_int64), ("filter_step_bytes", C.c_double),
        ("trace_estimate", C.c_double), ("p_used", C.c_int64),
        ("filter_kind", C.c_int32), ("filter_g", C.c_int32), ("filter_vpt", C.c_int32),
        ("filter_graph_replays", C.c_int64),
    ]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class apf_request_info(C.Structure):
    _fields_ = [
        ("status", C.c_int32), ("worker", C.c_int32),
        ("queue_ms", C.c_double), ("run_ms", C.c_double), ("latency_ms", C.c_double),
        ("footprint_bytes", C.c_int64),
    ]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class apf_server_info(C.Structure):
    _fields_ = [
        ("queued", C.c_int32), ("running", C.c_int32), ("peak_running", C.c_int32), ("workers", C.c_int32),
        ("in_flight_bytes", C.c_int64), ("peak_in_flight_bytes", C.c_int64), ("budget_bytes", C.c_int64),
        ("completed", C.c_int64), ("batched_launches", C.c_int64), ("widest_batch", C.c_int32),
        ("reserved", C.c_int32),
    ]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class ApfError(RuntimeError):
    def __init__(self, status, msg=""):
        super().__init__(f"apf status {status}: {msg}")
        self.status = status


_P = C.c_void_p
_D = C.c_double
_I32 = C.c_int32
_I64 = C.c_int64
_U64 = C.c_uint64
_DP = C.POINTER(C.c_double)

# name -> (restype, argtypes); the full exported surface of include/apf.h
SIGNATURES = {
    "apf_create": (_I32, [C.POINTER(_P), C.c_int, _P]),
    "apf_destroy": (_I32, [_P]),
    "apf_status_string": (C.c_char_p, [C.c_int]),
    "apf_last_error_message": (C.c_char_p, [_P]),
    "apf_launch_count": (_I64, [_P]),
    "apf_set_wait_limit": (_I32, [_P, _I64]),
    "apf_wait_probe": (_I32, [_P, _P, _I32]),
    "apf_matrix_create_csr": (_I32, [_P, _I64, _I64, _P, _P, _P, _I32, _I32, C.POINTER(_P)]),
    "apf_matrix_create_sell": (_I32, [_P, _I64, _I32, _I32, _P, _P, _P, _P, _P, _I32, C.POINTER(_P)]),
    "apf_matrix_destroy": (_I32, [_P]),
    "apf_matrix_info": (_I32, [_P, C.POINTER(_I64), C.POINTER(_I64), C.POINTER(_I32)]),
    "apf_params_default": (None, [C.POINTER(apf_params)]),
    "apf_solve": (_I32, [_P, _P, C.POINTER(apf_params), C.POINTER(_P)]),
    "apf_solve_slices": (_I32, [_P, _P, _I32, _P, _P, _P, C.POINTER(apf_params), C.POINTER(_P)]),
    "apf_result_slice_counts": (_I32, [_P, _I32, _P]),
    "apf_result_count": (_I32, [_P, C.POINTER(_I64)]),
    "apf_matrix_set_filter_kernel": (_I32, [_P, _I32, _I32, _I32]),
    "apf_server_create": (_I32, [C.POINTER(_P), _I32, _I32, _I64]),
    "apf_server_submit": (_I32, [_P, _I64, _I64, _P, _P, _P, _I32, C.POINTER(apf_params), C.POINTER(_I64)]),
    "apf_server_wait": (_I32, [_P, _I64, C.POINTER(_P), C.POINTER(apf_request_info)]),
    "apf_server_state": (_I32, [_P, C.POINTER(apf_server_info)]),
    "apf_server_destroy": (_I32, [_P]),
    "apf_result_eigvals": (_I32, [_P, _P]),
    "apf_result_eigvecs": (_I32, [_P, _P, _I64, _I32]),
    "apf_result_residuals": (_I32, [_P, _P]),
    "apf_result_stats": (_I32, [_P, C.POINTER(apf_stats)]),
    "apf_result_history": (_I32, [_P, _P, _I32, C.POINTER(_I32)]),
    "apf_result_destroy": (_I32, [_P]),
    "apf_filter_coefficients": (_I32, [_D, _D, _I32, _I32, _D, _P]),
    "apf_degree_select": (_I32, [_P, _I32, _I32, _P, _I32, _D, _D, _D, C.POINTER(_I32)]),
    "apf_spectrum_bounds": (_I32, [_P, _P, _I32, _U64, _D, _P]),
    "apf_count_estimate": (_I32, [_P, _P, _P, _I32, _D, _D, _I32, _I32, _U64, _DP]),
    "apf_filter_apply": (_I32, [_P, _P, _P, _I32, _D, _D, _I32, _P, _I64, _I64, _P, _I64]),
    "apf_filter_apply_defect": (_I32, [_P, _P, _P, _I32, _D, _D, _P, _P, _P, _I64, _I64, _P, _I64]),
    "apf_spmm": (_I32, [_P, _P, _P, _I64, _I64, _P, _I64]),
    "apf_gram": (_I32, [_P, _I32, _I64, _I64, _I64, _P, _I64, _P, _I64, _P, _I64]),
    "apf_gram_tc": (_I32, [_P, _I32, _I64, _I64, _I64, _P, _I64, _P, _I64, _P, _I64]),
    "apf_cholqr2": (_I32, [_P, _I32, _I64, _I64, _P, _I64]),
    "apf_block_update": (_I32, [_P, _I32, _I64, _I64, _I64, _P, _I64, _P, _I64, _P, _I64, _D, _D, _I32]),
    "apf_eigh_small": (_I32, [_P, _I32, _I64, _P, _I64, _P, _P, _I64]),
    "apf_rayleigh_ritz": (_I32, [_P, _P, _P, _I64, _I64, _P, _P, _I64]),
    "apf_residual_norms": (_I32, [_P, _P, _P, _I64, _I64, _P, _P]),
    "apf_random_block": (_I32, [_P, _I32, _U64, C.c_uint32, _I64, _I64, _P, _I64]),
    "apf_gram_noalloc": (_I32, [_I32, _I64, _I64, _I64, _P, _I64, _P, _I64, _P, _I64, _P]),
}


def _ptr(x):
    """Address of a numpy array, a torch tensor or None."""
    if x is None:
        return None
    if isinstance(x, np.ndarray):
        assert x.flags["C_CONTIGUOUS"]
        return x.ctypes.data
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    if isinstance(x, int):
        return x
    raise TypeError(type(x))


class Library:
    _inst = None

    def __init__(self, path=LIB_PATH):
        if not os.path.exists(path):
            raise RuntimeError(f"libapf.so is not built ({path}); run __graft_entry__.build()")
        self.lib = C.CDLL(path)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(self.lib, name)
            f.restype = res
            f.argtypes = args
        self.path = path

    @classmethod
    def load(cls, path=LIB_PATH):
        if cls._inst is None:
            cls._inst = cls(path)
        return cls._inst

    def __getattr__(self, name):
        if name.startswith("apf_"):
            return getattr(self.lib, name)
        raise AttributeError(name)

    def check(self, status, ctx=None):
        if status != APF_OK:
            msg = self.lib.apf_status_string(status).decode()
            if ctx is not None:
                msg += ": " + (self.lib.apf_last_error_message(ctx) or b"").decode()
            raise ApfError(status, msg)


# ---- object wrappers ---------------------------------------------------------------

class Context:
    """apf_create / apf_destroy; `stream` is a cudaStream_t handle (int) or None."""

    def __init__(self, device=0, stream=None, lib=None):
        self.lib = lib or Library.load()
        h = C.c_void_p()
        self.lib.check(self.lib.apf_create(C.byref(h), int(device), stream))
        self.h = h
        self._children = []

    def _adopt(self, obj):
        """Matrices and results must be freed before their context."""
        import weakref
        self._children = [r for r in self._children if r() is not None]
        self._children.append(weakref.ref(obj))

    def close(self):
        if self.h:
            for r in self._children:
                o = r()
                if o is not None:
                    o.close()
            self._children = []
            self.lib.apf_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def launch_count(self):
        return int(self.lib.apf_launch_count(self.h))

    def set_wait_limit(self, ns):
        """apf_set_wait_limit: time limit of the device-side waits (0: defaults)."""
        self.lib.check(self.lib.apf_set_wait_limit(self.h, int(ns)), self.h)

    def wait_probe(self, which, matrix=None):
        """apf_wait_probe: the status of a kernel whose wait nothing satisfies."""
        return int(self.lib.apf_wait_probe(self.h, matrix.h if matrix is not None else None, int(which)))


class Matrix:
    def __init__(self, ctx, h, n, dtype):
        self.ctx, self.h, self.n, self.dtype = ctx, h, n, dtype
        ctx._adopt(self)

    @classmethod
    def from_csr(cls, ctx, n, rowptr, colidx, vals, on_device=False):
        is_c = np.iscomplexobj(vals) if isinstance(vals, np.ndarray) else vals.is_complex()
        dt = APF_C128 if is_c else APF_R64
        if isinstance(vals, np.ndarray):
            rowptr = np.ascontiguousarray(rowptr, dtype=np.int64)
            colidx = np.ascontiguousarray(colidx, dtype=np.int32)
            vals = np.ascontiguousarray(vals, dtype=np.complex128 if is_c else np.float64)
        h = C.c_void_p()
        lib = ctx.lib
        lib.check(lib.apf_matrix_create_csr(ctx.h, int(n), int(colidx.shape[0]), _ptr(rowptr), _ptr(colidx),
                                            _ptr(vals), dt, 1 if on_device else 0, C.byref(h)), ctx.h)
        return cls(ctx, h, int(n), dt)

    @classmethod
    def from_sell(cls, ctx, n, Cw, sigma, perm, chunk_ptr, chunk_len, colidx, vals):
        is_c = np.iscomplexobj(vals)
        dt = APF_C128 if is_c else APF_R64
        perm = np.ascontiguousarray(perm, dtype=np.int64)
        chunk_ptr = np.ascontiguousarray(chunk_ptr, dtype=np.int64)
        chunk_len = np.ascontiguousarray(chunk_len, dtype=np.int32)
        colidx = np.ascontiguousarray(colidx, dtype=np.int32)
        vals = np.ascontiguousarray(vals, dtype=np.complex128 if is_c else np.float64)
        h = C.c_void_p()
        ctx.lib.check(ctx.lib.apf_matrix_create_sell(ctx.h, int(n), int(Cw), int(sigma), _ptr(perm), _ptr(chunk_ptr),
                                                     _ptr(chunk_len), _ptr(colidx), _ptr(vals), dt, C.byref(h)), ctx.h)
        return cls(ctx, h, int(n), dt)

    def set_filter_kernel(self, kind, G=0, VPT=0):
        """Pin the FP32 Clenshaw step kernel (0 = autotune, 1 = SELL, 2 = SELL two-step, 3 = CSR,
        4 = SELL column-tiled, 5 = column-tiled with near rows in shared memory); (G, VPT) = lanes per
        row x 16-byte vectors per lane, (0, 0) = default."""
        self.ctx.lib.check(self.ctx.lib.apf_matrix_set_filter_kernel(self.h, int(kind), int(G), int(VPT)))

    def close(self):
        if self.h and self.ctx.h:
            self.ctx.lib.apf_matrix_destroy(self.h)
        self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def info(self):
        n, nnz, dt = C.c_int64(), C.c_int64(), C.c_int32()
        self.ctx.lib.check(self.ctx.lib.apf_matrix_info(self.h, C.byref(n), C.byref(nnz), C.byref(dt)))
        return n.value, nnz.value, dt.value


def default_params(**kw) -> apf_params:
    lib = Library.load()
    p = apf_params()
    lib.apf_params_default(C.byref(p))
    for k, v in kw.items():
        if not hasattr(p, k):
            raise KeyError(k)
        setattr(p, k, v)
    return p


class Result:
    """Owns an apf_result; converts its contents to numpy."""

    def __init__(self, ctx, h, status):
        self.ctx, self.h, self.status = ctx, h, status
        ctx._adopt(self)

    def count(self):
        e = C.c_int64()
        self.ctx.lib.check(self.ctx.lib.apf_result_count(self.h, C.byref(e)))
        return e.value

    def eigvals(self):
        out = np.zeros(self.count())
        self.ctx.lib.check(self.ctx.lib.apf_result_eigvals(self.h, _ptr(out)))
        return out

    def residuals(self):
        out = np.zeros(self.count())
        self.ctx.lib.check(self.ctx.lib.apf_result_residuals(self.h, _ptr(out)))
        return out

    def eigvecs(self, n, is_complex, device_tensor=None):
        """n x e eigenvectors as a numpy array (column j for eigenvalue j), or
        into `device_tensor` (torch, shape (e, n): row j = column j, ld = n)."""
        e = self.count()
        if device_tensor is not None:
            self.ctx.lib.check(self.ctx.lib.apf_result_eigvecs(self.h, _ptr(device_tensor), int(n), 1), self.ctx.h)
            return device_tensor
        buf = np.zeros((e, n), dtype=np.complex128 if is_complex else np.float64)
        if e:
            self.ctx.lib.check(self.ctx.lib.apf_result_eigvecs(self.h, _ptr(buf), int(n), 0), self.ctx.h)
        return buf.T

    def stats(self):
        s = apf_stats()
        self.ctx.lib.check(self.ctx.lib.apf_result_stats(self.h, C.byref(s)))
        return s.as_dict()

    def slice_counts(self, nslices):
        """Pairs found per slice (apf_solve_slices results only)."""
        out = np.zeros(int(nslices), dtype=np.int64)
        self.ctx.lib.check(self.ctx.lib.apf_result_slice_counts(self.h, int(nslices), _ptr(out)))
        return out

    def history(self):
        cnt = C.c_int32()
        self.ctx.lib.check(self.ctx.lib.apf_result_history(self.h, None, 0, C.byref(cnt)))
        buf = np.zeros(max(1, cnt.value) * 6)
        self.ctx.lib.check(self.ctx.lib.apf_result_history(self.h, _ptr(buf), cnt.value, C.byref(cnt)))
        return [dict(zip(HISTORY_FIELDS, buf[6 * i:6 * i + 6])) for i in range(cnt.value)]

    def close(self):
        if self.h and (self.ctx.h or getattr(self.ctx, "owns_results", False)):
            self.ctx.lib.apf_result_destroy(self.h)
        self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def solve(ctx: Context, A: Matrix, params: apf_params, allow_no_convergence=False) -> Result:
    """apf_solve.  Raises ApfError on failure (NO_CONVERGENCE too, unless allowed)."""
    h = C.c_void_p()
    st = ctx.lib.apf_solve(ctx.h, A.h, C.byref(params), C.byref(h))
    if st == APF_ERR_NO_CONVERGENCE and allow_no_convergence:
        return Result(ctx, h, st)
    ctx.lib.check(st, ctx.h)
    return Result(ctx, h, st)


def solve_slices(ctx: Context, A: Matrix, a, b, p, params: apf_params, allow_no_convergence=False) -> Result:
    """apf_solve_slices over the intervals [a[s], b[s]] with subspace sizes p[s]."""
    a = np.ascontiguousarray(a, dtype=np.float64)
    b = np.ascontiguousarray(b, dtype=np.float64)
    p = np.ascontiguousarray(p, dtype=np.int64)
    if not (a.shape == b.shape == p.shape and a.ndim == 1):
        raise ValueError("a, b and p must be 1-d arrays of one length")
    h = C.c_void_p()
    st = ctx.lib.apf_solve_slices(ctx.h, A.h, int(a.size), _ptr(a), _ptr(b), _ptr(p), C.byref(params),
                                  C.byref(h))
    if st == APF_ERR_NO_CONVERGENCE and allow_no_convergence:
        return Result(ctx, h, st)
    ctx.lib.check(st, ctx.h)
    return Result(ctx, h, st)


class _RequestOwner:
    """Stands in for the context of a serving result: such a result owns its
    own native context, so it stays valid after the server is gone."""
    owns_results = True
    h = None

    def __init__(self, lib):
        self.lib = lib

    def _adopt(self, obj):
        pass


class Server:
    """apf_server_*: independent requests served with continuous batching on one device."""

    def __init__(self, device=0, max_concurrent=4, hbm_budget_bytes=0, lib=None):
        self.lib = lib or Library.load()
        h = C.c_void_p()
        self.lib.check(self.lib.apf_server_create(C.byref(h), int(device), int(max_concurrent),
                                                  int(hbm_budget_bytes)))
        self.h = h

    def submit(self, n, rowptr, colidx, vals, params):
        is_c = np.iscomplexobj(vals)
        rowptr = np.ascontiguousarray(rowptr, dtype=np.int64)
        colidx = np.ascontiguousarray(colidx, dtype=np.int32)
        vals = np.ascontiguousarray(vals, dtype=np.complex128 if is_c else np.float64)
        t = C.c_int64()
        self.lib.check(self.lib.apf_server_submit(self.h, int(n), int(colidx.shape[0]), _ptr(rowptr), _ptr(colidx),
                                                  _ptr(vals), APF_C128 if is_c else APF_R64, C.byref(params),
                                                  C.byref(t)))
        return t.value

    def wait(self, ticket, allow_no_convergence=False):
        """(Result or None, info dict) of a finished request."""
        h = C.c_void_p()
        info = apf_request_info()
        st = self.lib.apf_server_wait(self.h, int(ticket), C.byref(h), C.byref(info))
        res = Result(_RequestOwner(self.lib), h, st) if h.value else None
        if st != APF_OK and not (st == APF_ERR_NO_CONVERGENCE and allow_no_convergence):
            if res is not None:
                res.close()
            self.lib.check(st)
        return res, info.as_dict()

    def state(self):
        s = apf_server_info()
        self.lib.check(self.lib.apf_server_state(self.h, C.byref(s)))
        return s.as_dict()

    def close(self):
        if self.h:
            self.lib.apf_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---- the steps one by one ---------------------------------------------------------------

def filter_coefficients(am, bm, k, damping=APF_DAMP_LANCZOS_M, m_d=0.5):
    lib = Library.load()
    out = np.zeros(k + 1)
    lib.check(lib.apf_filter_coefficients(float(am), float(bm), int(k), int(damping), float(m_d), _ptr(out)))
    return out


def degree_select(ritz, e, coef, l1, l2, tau_a):
    lib = Library.load()
    ritz = np.ascontiguousarray(ritz, dtype=np.float64)
    coef = np.ascontiguousarray(coef, dtype=np.float64)
    d = C.c_int32()
    lib.check(lib.apf_degree_select(_ptr(ritz), ritz.size, int(e), _ptr(coef), coef.size - 1,
                                    float(l1), float(l2), float(tau_a), C.byref(d)))
    return d.value


def spectrum_bounds(ctx, A, steps=40, seed=20260401, pad=0.01):
    out = np.zeros(6)
    ctx.lib.check(ctx.lib.apf_spectrum_bounds(ctx.h, A.h, int(steps), int(seed), float(pad), _ptr(out)), ctx.h)
    return out


def count_estimate(ctx, A, coef, l1, l2, m, seed, precision=APF_FILTER_F64):
    """e~ = (1/m) sum_c z_c^H rho(l(A)) z_c over m seeded +-1 probes (Sec. 3.4)."""
    coef = np.ascontiguousarray(coef, dtype=np.float64)
    out = C.c_double()
    ctx.lib.check(ctx.lib.apf_count_estimate(ctx.h, A.h, _ptr(coef), coef.size - 1, float(l1), float(l2),
                                             int(precision), int(m), int(seed), C.byref(out)), ctx.h)
    return out.value


def filter_apply(ctx, A, coef, l1, l2, X, Y, precision=APF_FILTER_F64):
    """Y = rho(l(A)) X on device tensors X, Y of shape (n, p) (row-major)."""
    coef = np.ascontiguousarray(coef, dtype=np.float64)
    n, p = X.shape
    ctx.lib.check(ctx.lib.apf_filter_apply(ctx.h, A.h, _ptr(coef), coef.size - 1, float(l1), float(l2),
                                           int(precision), _ptr(X), X.stride(0), p, _ptr(Y), Y.stride(0)), ctx.h)
    return Y


def filter_apply_defect(ctx, A, coef, l1, l2, V, AV, lam, Y):
    coef = np.ascontiguousarray(coef, dtype=np.float64)
    n, p = V.shape
    ctx.lib.check(ctx.lib.apf_filter_apply_defect(ctx.h, A.h, _ptr(coef), coef.size - 1, float(l1), float(l2),
                                                  _ptr(V), _ptr(AV), _ptr(lam), V.stride(0), p, _ptr(Y),
                                                  Y.stride(0)), ctx.h)
    return Y


def spmm(ctx, A, X, Y):
    n, p = X.shape
    ctx.lib.check(ctx.lib.apf_spmm(ctx.h, A.h, _ptr(X), X.stride(0), p, _ptr(Y), Y.stride(0)), ctx.h)
    return Y


def gram(ctx, X, Y, G):
    n, pa = X.shape
    pb = Y.shape[1]
    dt = APF_C128 if X.is_complex() else APF_R64
    ctx.lib.check(ctx.lib.apf_gram(ctx.h, dt, n, pa, pb, _ptr(X), X.stride(0), _ptr(Y), Y.stride(0),
                                   _ptr(G), G.stride(0)), ctx.h)
    return G


def gram_tc(ctx, X, Y, G):
    """apf_gram_tc: G = X^H Y on the tensor cores (FP64-accurate slicing)."""
    n, pa = X.shape
    pb = Y.shape[1]
    dt = APF_C128 if X.is_complex() else APF_R64
    ctx.lib.check(ctx.lib.apf_gram_tc(ctx.h, dt, n, pa, pb, _ptr(X), X.stride(0), _ptr(Y), Y.stride(0),
                                      _ptr(G), G.stride(0)), ctx.h)
    return G


def block_update(ctx, X, M, Z, alpha=1.0, beta=0.0, tensor_cores=True):
    """apf_block_update: Z = beta Z + alpha X M on device tensors."""
    n, pa = X.shape
    pb = M.shape[1]
    dt = APF_C128 if X.is_complex() else APF_R64
    ctx.lib.check(ctx.lib.apf_block_update(ctx.h, dt, n, pa, pb, _ptr(X), X.stride(0), _ptr(M), M.stride(0),
                                           _ptr(Z), Z.stride(0), float(alpha), float(beta),
                                           1 if tensor_cores else 0), ctx.h)
    return Z


def cholqr2(ctx, X):
    n, p = X.shape
    dt = APF_C128 if X.is_complex() else APF_R64
    ctx.lib.check(ctx.lib.apf_cholqr2(ctx.h, dt, n, p, _ptr(X), X.stride(0)), ctx.h)
    return X


def eigh_small(ctx, B, w, U):
    p = B.shape[0]
    dt = APF_C128 if B.is_complex() else APF_R64
    ctx.lib.check(ctx.lib.apf_eigh_small(ctx.h, dt, p, _ptr(B), B.stride(0), _ptr(w), _ptr(U), U.stride(0)), ctx.h)
    return w, U


def rayleigh_ritz(ctx, A, Q, w, V):
    n, p = Q.shape
    ctx.lib.check(ctx.lib.apf_rayleigh_ritz(ctx.h, A.h, _ptr(Q), Q.stride(0), p, _ptr(w), _ptr(V), V.stride(0)),
                  ctx.h)
    return w, V


def residual_norms(ctx, A, V, w):
    n, p = V.shape
    out = np.zeros(p)
    ctx.lib.check(ctx.lib.apf_residual_norms(ctx.h, A.h, _ptr(V), V.stride(0), p, _ptr(w), _ptr(out)), ctx.h)
    return out


def random_block(ctx, seed, stream, X):
    n, p = X.shape
    dt = APF_C128 if X.is_complex() else APF_R64
    ctx.lib.check(ctx.lib.apf_random_block(ctx.h, dt, int(seed), int(stream), n, p, _ptr(X), X.stride(0)), ctx.h)
    return X
