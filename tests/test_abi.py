"""The C-ABI library loads and exports every entry point of include/apf.h
(no GPU needed: nothing here launches a kernel)."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_symbols():
    src = open(os.path.join(ROOT, "include", "apf.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(apf_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_2604_00914_gb300 import binding
    path = binding.LIB_PATH
    if not os.path.exists(path):
        import __graft_entry__
        __graft_entry__.build()
    return binding.Library.load()


def test_header_declares_the_boundary():
    names = _declared_symbols()
    for must in ("apf_create", "apf_destroy", "apf_matrix_create_csr", "apf_matrix_create_sell",
                 "apf_solve", "apf_result_eigvals", "apf_result_eigvecs", "apf_result_residuals",
                 "apf_result_stats", "apf_params_default", "apf_status_string", "apf_filter_apply"):
        assert must in names


def test_every_declared_symbol_is_exported(lib):
    for name in _declared_symbols():
        assert hasattr(lib.lib, name), name


def test_binding_covers_every_symbol(lib):
    from paper_2604_00914_gb300 import binding
    assert set(_declared_symbols()) == set(binding.SIGNATURES)


def test_struct_sizes_match_header(lib):
    """The ctypes mirrors have the C layout (checked through apf_params_default,
    which writes every field)."""
    from paper_2604_00914_gb300 import binding
    p = binding.apf_params()
    lib.apf_params_default(ctypes.byref(p))
    assert p.C == 1.4 and p.k_ratio == 2.5 and p.m_d == 0.5 and p.tau_a == 1e-3 and p.tau_c == 1e-10
    assert p.max_iter == 50 and p.lanczos_steps == 40 and p.spurious_rule == 1
    assert p.max_degree_cap == 100000 and p.init_block is None
    assert p.mu == 1.8 and p.trace_probes == 32 and p.filter_graphs == 1 and p.gram_tensor_cores == 1


def test_host_entry_points_without_gpu(lib):
    """The two host-only steps (coefficients, Alg. 3) run without a device; they
    are checked against the oracle in the GPU-free suite as well."""
    from oracle import chebyshev as cb
    from paper_2604_00914_gb300 import binding
    for damp, name, m in ((binding.APF_DAMP_LANCZOS_M, cb.DAMP_LANCZOS_M, 0.5),
                          (binding.APF_DAMP_JACKSON, cb.DAMP_JACKSON, 0.5),
                          (binding.APF_DAMP_NONE, cb.DAMP_NONE, 0.5)):
        a = binding.filter_coefficients(-0.2, 0.35, 300, damp, m)
        ref = cb.filter_coefficients(-0.2, 0.35, 300, name, m)
        assert np.max(np.abs(a - ref)) < 1e-14
    coef = cb.filter_coefficients(-0.05, 0.05, 600)
    ritz = np.concatenate([np.linspace(-0.04, 0.04, 6), np.linspace(0.08, 0.2, 6)])
    assert binding.degree_select(ritz, 6, coef, 1.0, 0.0, 1e-3) == cb.degree_select(ritz, 6, coef, 1.0, 0.0, 1e-3)
    assert binding.degree_select(ritz, 12, coef, 1.0, 0.0, 1e-3) == 600


def test_status_strings(lib):
    assert lib.apf_status_string(0) == b"ok"
    assert b"Hermitian" in lib.apf_status_string(4)
    assert lib.apf_status_string(99) == b"unknown status"


def test_argument_errors_without_device(lib):
    from paper_2604_00914_gb300 import binding
    out = np.zeros(10)
    # interval outside (-1, 1) or reversed
    assert lib.apf_filter_coefficients(0.3, 0.2, 9, 0, 0.5, out.ctypes.data) == binding.APF_ERR_ARG
    assert lib.apf_filter_coefficients(-1.5, 0.2, 9, 0, 0.5, out.ctypes.data) == binding.APF_ERR_ARG
    assert lib.apf_solve(None, None, None, None) == binding.APF_ERR_ARG
    # the entry points beyond one solve reject missing handles before any device work
    import ctypes
    h = ctypes.c_void_p()
    cnt = np.zeros(4, dtype=np.int64)
    assert lib.apf_solve_slices(None, None, 1, None, None, None, None, None) == binding.APF_ERR_ARG
    assert lib.apf_result_slice_counts(None, 1, cnt.ctypes.data) == binding.APF_ERR_ARG
    assert lib.apf_count_estimate(None, None, None, 4, 0.1, 0.0, 0, 8, 1, None) == binding.APF_ERR_ARG
    assert lib.apf_matrix_set_filter_kernel(None, 1, 0, 0) == binding.APF_ERR_ARG
    assert lib.apf_server_create(None, 0, 2, 0) == binding.APF_ERR_ARG
    assert lib.apf_server_create(ctypes.byref(h), 0, 0, 0) == binding.APF_ERR_ARG  # no worker slot
    assert lib.apf_server_create(ctypes.byref(h), 0, 65, 0) == binding.APF_ERR_ARG
    assert lib.apf_server_submit(None, 10, 0, None, None, None, 0, None, None) == binding.APF_ERR_ARG
    assert lib.apf_server_wait(None, 1, ctypes.byref(h), None) == binding.APF_ERR_ARG
    assert lib.apf_server_state(None, None) == binding.APF_ERR_ARG
    assert lib.apf_server_destroy(None) == binding.APF_OK
