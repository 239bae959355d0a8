"""GB300 (sm_103a) sliding-window median filter -- Python binding of libmf.so.

The library implements "Median Filtering is Equivalent to Sorting"
(Suomela): phase 1 sorts each length-k block, phase 2 post-processes every
adjacent block pair with two sorted doubly-linked lists (dancing links).
All arithmetic runs in the CUDA kernels of ``libmf.so``; this module only
marshals arguments (tensor pointers, sizes, streams) into the C ABI declared
in ``include/mf.h`` and turns status codes into exceptions.  There is no CPU
fallback: if the library is missing, every call raises.

Functions carry the C names: ``mf_create``, ``mf_set_stream``, ``mf_filter``,
``mf_filter_host``, ``mf_filter_batched``, ``mf_filter_backward``,
``mf_filter_noalloc``, ``mf_sync``, ``mf_launch_count``, ``mf_set_tuning``, ``mf_set_timing``,
``mf_kernel_times``, ``mf_debug_take``, ``mf_debug_selftest``, ``mf_status_str``, ``mf_destroy``.
With MF_DEBUG=1 in the environment the debug build ``libmf_debug.so`` is
loaded instead (device checks of indices and list invariants).
``median_filter`` is a convenience wrapper that allocates the outputs.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
# MF_DEBUG=1 selects the debug build (device checks; mf_debug_take), made by
# paper_1406_1717_gb300.build.build(debug=True)
DEBUG = os.environ.get("MF_DEBUG", "") not in ("", "0")
LIB_PATH = os.path.join(_PKG, "libmf_debug.so" if DEBUG else "libmf.so")

MF_INT32, MF_FLOAT32, MF_INT64, MF_FLOAT64 = 0, 1, 2, 3

STATUS_NAMES = {
    0: "MF_OK", 1: "MF_ERR_NULL", 2: "MF_ERR_BAD_N", 3: "MF_ERR_EVEN_K",
    4: "MF_ERR_K_GT_N", 5: "MF_ERR_DTYPE", 6: "MF_ERR_OOM", 7: "MF_ERR_CUDA",
    8: "MF_ERR_UNSUPPORTED", 9: "MF_ERR_OVERLAP", 10: "MF_ERR_DEVICE",
    11: "MF_ERR_BAD_SEGMENT", 12: "MF_ERR_TOO_LARGE", 13: "MF_ERR_BAD_RANK",
}

# mf_segment: int64 x_off, int64 n, int64 y_off, int32 k, int32 pad
SEGMENT_DTYPE = np.dtype([("x_off", "<i8"), ("n", "<i8"), ("y_off", "<i8"),
                          ("k", "<i4"), ("pad", "<i4")])


class MFError(RuntimeError):
    def __init__(self, status: int, what: str = ""):
        self.status = status
        super().__init__(f"{what}: {mf_status_str(status)}" if what else mf_status_str(status))


_lock = threading.Lock()
_lib = None


def load_library(path: str = LIB_PATH):
    """Load libmf.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(path):
            how = ("paper_1406_1717_gb300.build.build(debug=True)" if path.endswith("_debug.so")
                   else "__graft_entry__.build() or python -m paper_1406_1717_gb300.build")
            raise RuntimeError(f"{path} is missing: build it with {how}")
        lib = ctypes.CDLL(path)
        c = ctypes
        vp, i32, i64, sz = c.c_void_p, c.c_int32, c.c_int64, c.c_size_t
        sig = {
            "mf_create": ([c.POINTER(vp), c.c_int, vp, sz], c.c_int),
            "mf_set_stream": ([vp, vp], c.c_int),
            "mf_filter": ([vp, c.c_int, vp, i64, i32, vp, vp], c.c_int),
            "mf_filter_host": ([vp, c.c_int, vp, i64, i32, vp, vp], c.c_int),
            "mf_filter_rank": ([vp, c.c_int, vp, i64, i32, i32, vp, vp], c.c_int),
            "mf_filter_batched": ([vp, c.c_int, vp, vp, vp, i32, vp], c.c_int),
            "mf_filter_backward": ([vp, vp, vp, i64, i32, vp], c.c_int),
            "mf_filter_backward_rows": ([vp, vp, vp, i64, i64, i32, vp], c.c_int),
            "mf_filter_noalloc": ([c.c_int, vp, i64, i32, vp, vp, vp], c.c_int),
            "mf_sync": ([vp], c.c_int),
            "mf_launch_count": ([vp, c.POINTER(c.c_uint64)], c.c_int),
            "mf_debug_take": ([vp, c.POINTER(c.c_uint32), c.POINTER(c.c_uint32),
                               c.POINTER(c.c_uint64)], c.c_int),
            "mf_debug_selftest": ([vp], c.c_int),
            "mf_set_timing": ([vp, c.c_int], c.c_int),
            "mf_set_tuning": ([vp, i32, i32, i32], c.c_int),
            "mf_set_sort_variant": ([vp, i32, i32], c.c_int),
            "mf_set_tier_threshold": ([vp, i32], c.c_int),
            "mf_get_tier_threshold": ([vp, c.POINTER(i32)], c.c_int),
            "mf_batched_workspace_bytes": ([vp, c.c_int, vp, i32, c.POINTER(sz)], c.c_int),
            "mf_workspace_size": ([vp, c.POINTER(sz)], c.c_int),
            "mf_release_workspace": ([vp], c.c_int),
            "mf_fill_splitmix": ([c.c_int, vp, i64, c.c_uint64, vp], c.c_int),
            "mf_kernel_times": ([vp, i32, c.POINTER(c.c_float)], c.c_int),
            "mf_status_str": ([c.c_int], c.c_char_p),
            "mf_destroy": ([vp], c.c_int),
        }
        for name, (args, res) in sig.items():
            fn = getattr(lib, name)
            fn.argtypes = args
            fn.restype = res
        _lib = lib
        return lib


def _check(status: int, what: str):
    if status != 0:
        raise MFError(status, what)


def _dtype_code(t) -> int:
    import torch
    code = {torch.int32: MF_INT32, torch.float32: MF_FLOAT32,
            torch.int64: MF_INT64, torch.float64: MF_FLOAT64}.get(t.dtype)
    if code is not None:
        return code
    raise TypeError(f"median filter supports int32, float32, int64 and float64, got {t.dtype}")


def _dptr(t, name: str):
    if t is None:
        return None
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    return ctypes.c_void_p(t.data_ptr())


def _stream_ptr(stream):
    if stream is None:
        return None
    if hasattr(stream, "cuda_stream"):
        return ctypes.c_void_p(stream.cuda_stream)
    return ctypes.c_void_p(int(stream))


# ---------------------------------------------------------------------------
# C-ABI functions
# ---------------------------------------------------------------------------
def mf_status_str(status: int) -> str:
    try:
        return load_library().mf_status_str(int(status)).decode()
    except RuntimeError:
        return STATUS_NAMES.get(int(status), f"status {status}")


def mf_create(device: int = 0, stream=None, max_workspace_bytes: int = 0):
    """Create a handle on CUDA device ``device`` bound to ``stream`` (torch
    stream, raw cudaStream_t int, or None for the default stream)."""
    h = ctypes.c_void_p()
    _check(load_library().mf_create(ctypes.byref(h), int(device), _stream_ptr(stream),
                                    int(max_workspace_bytes)), "mf_create")
    return h


def mf_set_stream(handle, stream):
    _check(load_library().mf_set_stream(handle, _stream_ptr(stream)), "mf_set_stream")


def mf_filter(handle, x, k: int, y, argmed=None):
    """y[i] = median(x[i .. i+k-1]) on the device; x, y (and argmed, int32)
    are contiguous CUDA tensors of the handle's device."""
    _check(load_library().mf_filter(handle, _dtype_code(x), _dptr(x, "x"), x.numel(), int(k),
                                    _dptr(y, "y"), _dptr(argmed, "argmed")), "mf_filter")


def mf_filter_rank(handle, x, k: int, rank: int, y, argmed=None):
    """y[i] = the element of 0-based rank `rank` in x[i .. i+k-1] (any k >= 1;
    even k with rank = k//2 - 1 is the lower median)."""
    _check(load_library().mf_filter_rank(handle, _dtype_code(x), _dptr(x, "x"), x.numel(),
                                         int(k), int(rank), _dptr(y, "y"),
                                         _dptr(argmed, "argmed")), "mf_filter_rank")


def mf_filter_host(handle, x, k: int, y, argmed=None):
    """Same as mf_filter with HOST arrays (numpy or CPU tensors); synchronous."""
    def hptr(a):
        if a is None:
            return None
        if isinstance(a, np.ndarray):
            if not a.flags["C_CONTIGUOUS"]:
                raise ValueError("host arrays must be contiguous")
            return ctypes.c_void_p(a.ctypes.data)
        return _dptr(a, "host tensor")
    if isinstance(x, np.ndarray):
        code = {np.dtype(np.int32): MF_INT32, np.dtype(np.float32): MF_FLOAT32,
                np.dtype(np.int64): MF_INT64, np.dtype(np.float64): MF_FLOAT64}.get(x.dtype)
        if code is None:
            raise TypeError(f"median filter supports int32, float32, int64 and float64, got {x.dtype}")
        n = x.size
    else:
        code, n = _dtype_code(x), x.numel()
    _check(load_library().mf_filter_host(handle, code, hptr(x), n, int(k), hptr(y), hptr(argmed)),
           "mf_filter_host")


def make_segments(n, k, x_off, y_off) -> np.ndarray:
    segs = np.zeros(len(n), dtype=SEGMENT_DTYPE)
    segs["n"], segs["k"], segs["x_off"], segs["y_off"] = n, k, x_off, y_off
    return segs


def mf_filter_batched(handle, x, y, segs: np.ndarray, argmed=None):
    """Filter many signals packed in x; ``segs`` is a numpy array of SEGMENT_DTYPE."""
    segs = np.ascontiguousarray(segs, dtype=SEGMENT_DTYPE)
    _check(load_library().mf_filter_batched(handle, _dtype_code(x), _dptr(x, "x"), _dptr(y, "y"),
                                            ctypes.c_void_p(segs.ctypes.data), int(segs.size),
                                            _dptr(argmed, "argmed")), "mf_filter_batched")


def mf_filter_backward(handle, gy, argmed, n: int, k: int, gx):
    """gx[j] = sum of gy[i] over argmed[i] == j (float32 tensors, int32 argmed)."""
    _check(load_library().mf_filter_backward(handle, _dptr(gy, "gy"), _dptr(argmed, "argmed"),
                                             int(n), int(k), _dptr(gx, "gx")),
           "mf_filter_backward")


def mf_filter_backward_rows(handle, gy, argmed, rows: int, n: int, k: int, gx):
    """mf_filter_backward of ``rows`` equal-length rows in one launch
    (row-major gy / argmed of rows x (n-k+1), gx of rows x n)."""
    _check(load_library().mf_filter_backward_rows(handle, _dptr(gy, "gy"), _dptr(argmed, "argmed"),
                                                  int(rows), int(n), int(k), _dptr(gx, "gx")),
           "mf_filter_backward_rows")


def mf_filter_noalloc(x, k: int, y, argmed=None, stream=None):
    """mf_filter without a handle and without any device allocation (scratch
    is a fixed array inside the library); for callers that cannot allocate."""
    _check(load_library().mf_filter_noalloc(_dtype_code(x), _dptr(x, "x"), x.numel(), int(k),
                                            _dptr(y, "y"), _dptr(argmed, "argmed"),
                                            _stream_ptr(stream)), "mf_filter_noalloc")


def mf_sync(handle):
    _check(load_library().mf_sync(handle), "mf_sync")


def mf_launch_count(handle) -> int:
    c = ctypes.c_uint64()
    _check(load_library().mf_launch_count(handle, ctypes.byref(c)), "mf_launch_count")
    return int(c.value)


def mf_debug_take(handle):
    """Debug build: (failed checks, first site, first value) since the last
    take, after all work on the device finished; the records are cleared.
    Raises MFError(MF_ERR_UNSUPPORTED) in the normal build."""
    cnt, site, val = ctypes.c_uint32(), ctypes.c_uint32(), ctypes.c_uint64()
    _check(load_library().mf_debug_take(handle, ctypes.byref(cnt), ctypes.byref(site),
                                        ctypes.byref(val)), "mf_debug_take")
    return int(cnt.value), int(site.value), int(val.value)


def mf_debug_selftest(handle):
    """Debug build: one device thread fails one check (site 999, value 42)."""
    _check(load_library().mf_debug_selftest(handle), "mf_debug_selftest")


KERNEL_NAMES = ("sort", "unwind", "chain", "store")


def mf_set_tuning(handle, k: int, sort_pairs_per_cta: int = 0, store_pairs_per_cta: int = 0):
    """Launch-plan choice for the window-size class containing k (0 = built-in)."""
    _check(load_library().mf_set_tuning(handle, int(k), int(sort_pairs_per_cta),
                                        int(store_pairs_per_cta)), "mf_set_tuning")


def mf_set_sort_variant(handle, k: int, variant: int = 0):
    """Block-sort variant for the class containing k: 0 built-in, 1 merge-sort
    tiles (fused path), 2 warp radix sort (four-kernel path), 3 merge-sort
    tiles that skip tiles of ordered blocks."""
    _check(load_library().mf_set_sort_variant(handle, int(k), int(variant)), "mf_set_sort_variant")


def mf_set_tier_threshold(handle, k_large_from: int = 0):
    """Calls with k >= k_large_from use the large-k tier (0 = the pipeline's limit)."""
    _check(load_library().mf_set_tier_threshold(handle, int(k_large_from)),
           "mf_set_tier_threshold")


def mf_get_tier_threshold(handle) -> int:
    out = ctypes.c_int32()
    _check(load_library().mf_get_tier_threshold(handle, ctypes.byref(out)), "mf_get_tier_threshold")
    return int(out.value)


def tier_of(handle, k: int) -> str:
    """"large" if calls with window k on this handle run the large-k tier, else "pipeline"."""
    return "large" if int(k) >= mf_get_tier_threshold(handle) else "pipeline"


def mf_batched_workspace_bytes(handle, segs: np.ndarray, dtype: int = MF_FLOAT32) -> int:
    """Workspace bytes mf_filter_batched needs for these descriptors on this
    handle (dtype: MF_INT32, MF_FLOAT32, MF_INT64 or MF_FLOAT64)."""
    segs = np.ascontiguousarray(segs, dtype=SEGMENT_DTYPE)
    out = ctypes.c_size_t()
    _check(load_library().mf_batched_workspace_bytes(handle, int(dtype), segs.ctypes.data,
                                                     len(segs), ctypes.byref(out)),
           "mf_batched_workspace_bytes")
    return int(out.value)


def mf_workspace_size(handle) -> int:
    out = ctypes.c_size_t()
    _check(load_library().mf_workspace_size(handle, ctypes.byref(out)), "mf_workspace_size")
    return int(out.value)


def mf_release_workspace(handle):
    _check(load_library().mf_release_workspace(handle), "mf_release_workspace")


def mf_fill_splitmix(x, seed: int, stream=None):
    """Fill the CUDA tensor x (int32 or float32) with SplitMix64 payload samples."""
    import torch
    if not x.is_cuda or not x.is_contiguous():
        raise TypeError("x must be a contiguous CUDA tensor")
    s = stream if stream is not None else torch.cuda.current_stream(x.device)
    _check(load_library().mf_fill_splitmix(_dtype_code(x), x.data_ptr(), x.numel(),
                                           int(seed) & 0xFFFFFFFFFFFFFFFF, s.cuda_stream),
           "mf_fill_splitmix")


def mf_set_timing(handle, enable: bool = True):
    _check(load_library().mf_set_timing(handle, 1 if enable else 0), "mf_set_timing")


def mf_kernel_times(handle, ncalls: int) -> dict:
    """Per-kernel milliseconds summed over the last ``ncalls`` timed calls."""
    arr = (ctypes.c_float * 4)()
    _check(load_library().mf_kernel_times(handle, int(ncalls), arr), "mf_kernel_times")
    return dict(zip(KERNEL_NAMES, [float(v) for v in arr]))


def mf_destroy(handle):
    _check(load_library().mf_destroy(handle), "mf_destroy")


# ---------------------------------------------------------------------------
# convenience
# ---------------------------------------------------------------------------
_handles = {}


def default_handle(device: int):
    """One handle per device, bound to the default stream; call sites rebind
    it to torch's current stream before use."""
    h = _handles.get(device)
    if h is None:
        h = mf_create(device)
        _handles[device] = h
    return h


def median_filter(x, k: int, return_argmed: bool = False):
    """Median filter of a 1-D CUDA tensor on torch's current stream."""
    import torch
    if x.dim() != 1 or not x.is_cuda:
        raise ValueError("x must be a 1-D CUDA tensor")
    dev = x.device.index
    h = default_handle(dev)
    mf_set_stream(h, torch.cuda.current_stream(x.device))
    m = x.numel() - int(k) + 1
    if m < 1:
        raise ValueError("need k <= len(x)")
    y = torch.empty(m, dtype=x.dtype, device=x.device)
    a = torch.empty(m, dtype=torch.int32, device=x.device) if return_argmed else None
    mf_filter(h, x.contiguous(), k, y, a)
    return (y, a) if return_argmed else y
