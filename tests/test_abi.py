"""The C-ABI library loads and exports every function include/*.h declares
(no GPU needed: nothing is called that touches a device)."""
import ctypes
import os

import pytest

from paper_1409_5000_gb300 import _build, binding


@pytest.fixture(scope="module")
def libcb():
    if not os.path.exists(_build.cb_lib_path()):
        _build.build_cb()
    return ctypes.CDLL(_build.cb_lib_path())


def test_header_declares_the_boundary():
    names = set(binding.declared_functions())
    for required in ["cb_graph_upload", "cb_graph_free", "cb_communicability",
                     "cb_ensemble_scores", "cb_topk", "cb_last_error", "cb_version"]:
        assert required in names


def test_every_declared_symbol_is_exported(libcb):
    missing = [n for n in binding.declared_functions() if not hasattr(libcb, n)]
    assert not missing, missing


def test_binding_wraps_every_declared_function():
    """The Python binding mirrors the C ABI name for name."""
    missing = [n for n in binding.declared_functions() if not callable(getattr(binding, n, None))]
    assert not missing, missing


def test_version_and_error_string(libcb):
    libcb.cb_version.restype = ctypes.c_uint32
    assert libcb.cb_version() >> 16 == 1
    libcb.cb_last_error.restype = ctypes.c_char_p
    assert isinstance(libcb.cb_last_error(), bytes)


def test_argument_errors_need_no_device(libcb):
    """Host-side argument checks reject bad calls before any CUDA call."""
    L = binding.lib()
    assert L.cb_topk(None, 10, 3, None, None, None) == binding.CB_ERR_ARG
    assert L.cb_graph_free(None) == binding.CB_ERR_ARG
    out = ctypes.c_void_p()
    assert L.cb_graph_upload(0, None, None, None, None, 0, None, ctypes.byref(out)) == binding.CB_ERR_ARG
    # an unknown upload flag is rejected before the arrays are looked at
    n = (ctypes.c_uint32 * 1)(4)
    nnz = (ctypes.c_uint64 * 1)(0)
    rp = (ctypes.c_uint32 * 5)()
    rpp = (ctypes.c_void_p * 1)(ctypes.addressof(rp))
    unknown = 16
    assert unknown & (binding.CB_VALIDATE | binding.CB_DEVICE_PTRS | binding.CB_CSR_ONLY
                      | binding.CB_TWO_PHASE) == 0
    assert L.cb_graph_upload(1, n, nnz, rpp, rpp, unknown, None, ctypes.byref(out)) == binding.CB_ERR_ARG
    assert b"unknown flag" in L.cb_last_error()
    both = binding.CB_CSR_ONLY | binding.CB_TWO_PHASE
    assert L.cb_graph_upload(1, n, nnz, rpp, rpp, both, None, ctypes.byref(out)) == binding.CB_ERR_ARG
    assert b"exclude each other" in L.cb_last_error()
    assert L.cb_communicability(None, 0, 10, 0, None, None, None, None) == binding.CB_ERR_ARG
    assert L.cb_ensemble_scores(None, 10, 0, 5, None, None, None, None) == binding.CB_ERR_ARG
    assert b"null" in L.cb_last_error()


def test_debug_library_exports_the_same_symbols():
    """libcb_debug.so (-DCB_DEBUG) exports every declared function and says
    which build it is; the release build says 0 and reports no violations
    without touching a device."""
    path = _build.cb_lib_path(debug=True)
    if not os.path.exists(path):
        _build.build_cb(debug=True)
    dbg = ctypes.CDLL(path)
    missing = [n for n in binding.declared_functions() if not hasattr(dbg, n)]
    assert not missing, missing
    dbg.cb_debug_build.restype = ctypes.c_uint32
    assert dbg.cb_debug_build() == 1
    L = binding.lib()
    assert binding.cb_debug_build() == (1 if os.environ.get("CB_DEBUG") == "1" else 0)
    if not binding.cb_debug_build():
        assert binding.cb_debug_violations() == (0, 0)
    assert L.cb_debug_violations(None, None, 0) == binding.CB_ERR_ARG
