"""Host-side checks of the C ABI (no GPU needed, no compute calls).

* the library loads and exports every function that include/mf.h declares;
* status strings; NULL-handle and argument errors are reported before any
  CUDA work is enqueued;
* segment descriptor layout matches the C struct.
"""
import ctypes
import os
import re

import numpy as np
import pytest

import paper_1406_1717_gb300 as mf
from paper_1406_1717_gb300 import build as mfbuild

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    mfbuild.build()
    return mf.load_library()


def declared_functions():
    inc = os.path.join(ROOT, "include")
    text = "".join(open(os.path.join(inc, f)).read() for f in sorted(os.listdir(inc))
                   if f.endswith(".h"))
    return sorted(set(re.findall(r"^\s*(?:mf_status|const char\*)\s+(mf_\w+)\s*\(", text, re.M)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("mf_create", "mf_filter", "mf_filter_batched", "mf_filter_backward",
                     "mf_sync", "mf_status_str", "mf_destroy", "mf_filter_host"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name
        assert isinstance(getattr(lib, name), ctypes._CFuncPtr)


def test_status_strings(lib):
    for code, name in mf.STATUS_NAMES.items():
        assert mf.mf_status_str(code).startswith(name)
    assert mf.mf_status_str(12345) == "MF_ERR_UNKNOWN"


def test_null_handle_rejected_without_cuda(lib):
    vp = ctypes.c_void_p
    assert lib.mf_filter(None, 0, vp(16), 10, 3, vp(64), None) == 1
    assert lib.mf_filter_host(None, 0, vp(16), 10, 3, vp(64), None) == 1
    assert lib.mf_filter_batched(None, 0, vp(16), vp(64), vp(128), 1, None) == 1
    assert lib.mf_filter_backward(None, vp(16), vp(32), 10, 3, vp(64)) == 1
    assert lib.mf_filter_backward_rows(None, vp(16), vp(32), 2, 10, 3, vp(64)) == 1
    assert lib.mf_sync(None) == 1
    assert lib.mf_destroy(None) == 1
    assert lib.mf_set_stream(None, None) == 1
    assert lib.mf_create(None, 0, None, 0) == 1


def test_create_reports_missing_or_wrong_device(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    h = ctypes.c_void_p()
    assert lib.mf_create(ctypes.byref(h), 0, None, 0) == 10     # MF_ERR_DEVICE
    assert h.value is None


def test_segment_dtype_matches_c_struct():
    assert mf.SEGMENT_DTYPE.itemsize == 32
    segs = mf.make_segments([10, 20], [3, 5], [0, 10], [0, 8])
    raw = segs.tobytes()
    assert np.frombuffer(raw[:8], "<i8")[0] == 0
    assert np.frombuffer(raw[8:16], "<i8")[0] == 10
    assert np.frombuffer(raw[24:28], "<i4")[0] == 3
    assert np.frombuffer(raw[32 + 8:32 + 16], "<i8")[0] == 20


def test_binding_refuses_missing_library(tmp_path):
    # the binding never falls back to CPU code: a missing library is an error
    saved = mf._lib
    try:
        mf._lib = None
        with pytest.raises(RuntimeError):
            mf.load_library(str(tmp_path / "missing.so"))
    finally:
        mf._lib = saved


def test_debug_entries_check_their_arguments(lib):
    vp = ctypes.c_void_p
    c, s, v = ctypes.c_uint32(7), ctypes.c_uint32(7), ctypes.c_uint64(7)
    assert lib.mf_debug_take(None, ctypes.byref(c), ctypes.byref(s), ctypes.byref(v)) == 1
    assert lib.mf_debug_selftest(None) == 1


def test_debug_build_compiles_and_exports_the_boundary():
    """The MF_DEBUG build (device checks that record and clamp) compiles for
    sm_103a and exports the same functions; it is loaded here without being
    called (no GPU)."""
    path = mfbuild.build(debug=True)
    assert path.endswith("libmf_debug.so") and os.path.exists(path)
    dbg = ctypes.CDLL(path)
    for name in declared_functions():
        assert hasattr(dbg, name), name
