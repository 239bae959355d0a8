"""CPU oracle for the sliding-window median filter -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline /
reference arm may import this package.  The CUDA library in
``paper_1406_1717_gb300/`` never imports it and shares no code with it.

``mf_oracle.c`` is the plain definition (paper Section 1: y_i is the median of
x_i .. x_{i+k-1}; Section 2: find the median of every window separately),
compiled with gcc into ``oracle/_build/liboracle.so`` on first use.
``paper_method.py`` is a set-level model of the paper's method, written from
its definitions (the block interface of Section 5, the list equations of
Section 4, the post-processing steps of Section 6.2), for the invariant and
case-table tests; it is not used to produce expected values for the CUDA
path.

Parity pins: every function here is checked in ``tests/test_oracle_pins.py``
against brute force, closed forms, library routines (numpy / scipy), the
paper's lower-bound reduction (Section 2) and IEEE totalOrder fixtures.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mf_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

INT32, FLOAT32, INT64, FLOAT64 = 0, 1, 2, 3


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (OpenMP if available). Returns the .so path."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    base = ["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-o", tmp, _SRC]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True,
                       capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            lib.mfo_filter.argtypes = [ctypes.c_int, ctypes.c_void_p, ctypes.c_int64,
                                       ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p,
                                       ctypes.c_int]
            lib.mfo_filter.restype = ctypes.c_int
            lib.mfo_windows.argtypes = [ctypes.c_int, ctypes.c_void_p, ctypes.c_int64,
                                        ctypes.c_int32, ctypes.c_void_p, ctypes.c_int64,
                                        ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int]
            lib.mfo_windows.restype = ctypes.c_int
            lib.mfo_rank_filter.argtypes = [ctypes.c_int, ctypes.c_void_p, ctypes.c_int64,
                                            ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p,
                                            ctypes.c_void_p, ctypes.c_int]
            lib.mfo_rank_filter.restype = ctypes.c_int
            lib.mfo_rank_windows.argtypes = [ctypes.c_int, ctypes.c_void_p, ctypes.c_int64,
                                             ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p,
                                             ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p,
                                             ctypes.c_int]
            lib.mfo_rank_windows.restype = ctypes.c_int
            lib.mfo_max_threads.argtypes = []
            lib.mfo_max_threads.restype = ctypes.c_int
            _lib = lib
    return _lib


def _dtype_code(x: np.ndarray) -> int:
    code = {np.dtype(np.int32): INT32, np.dtype(np.float32): FLOAT32,
            np.dtype(np.int64): INT64, np.dtype(np.float64): FLOAT64}.get(x.dtype)
    if code is None:
        raise TypeError(f"oracle supports int32, float32, int64 and float64, got {x.dtype}")
    return code


def max_threads() -> int:
    return int(_load().mfo_max_threads())


def median_filter(x: np.ndarray, k: int, nthreads: int = 0, with_arg: bool = True):
    """y[i] = median(x[i .. i+k-1]) for i in 0..n-k; returns (y, argmed or None).

    y has x's dtype and carries the median element's exact bits; argmed is the
    int64 index of that element (rank h under the (value, index) order).
    """
    x = np.ascontiguousarray(x)
    code = _dtype_code(x)
    n = x.size
    if k < 1 or k % 2 == 0 or k > n:
        raise ValueError(f"need odd 1 <= k <= n, got n={n} k={k}")
    m = n - k + 1
    y = np.empty(m, dtype=x.dtype)
    arg = np.empty(m, dtype=np.int64) if with_arg else None
    rc = _load().mfo_filter(code, x.ctypes.data, n, k, y.ctypes.data,
                            arg.ctypes.data if with_arg else None, nthreads)
    if rc != 0:
        raise ValueError(f"mfo_filter returned {rc}")
    return y, arg


def window_medians(x: np.ndarray, k: int, starts, nthreads: int = 0):
    """Medians of the windows x[s .. s+k-1] for each s in ``starts``."""
    x = np.ascontiguousarray(x)
    code = _dtype_code(x)
    starts = np.ascontiguousarray(np.asarray(starts, dtype=np.int64))
    y = np.empty(starts.size, dtype=x.dtype)
    arg = np.empty(starts.size, dtype=np.int64)
    rc = _load().mfo_windows(code, x.ctypes.data, x.size, k, starts.ctypes.data,
                             starts.size, y.ctypes.data, arg.ctypes.data, nthreads)
    if rc != 0:
        raise ValueError(f"mfo_windows returned {rc}")
    return y, arg


def rank_filter(x: np.ndarray, k: int, r: int, nthreads: int = 0):
    """y[i] = element of 0-based rank r in x[i .. i+k-1] (any k >= 1); (y, arg).

    The median of an odd window is r = (k-1)/2; the lower median of an even
    window r = k/2 - 1."""
    x = np.ascontiguousarray(x)
    code = _dtype_code(x)
    n = x.size
    if k < 1 or k > n or not 0 <= r < k:
        raise ValueError(f"need 1 <= k <= n and 0 <= r < k, got n={n} k={k} r={r}")
    m = n - k + 1
    y = np.empty(m, dtype=x.dtype)
    arg = np.empty(m, dtype=np.int64)
    rc = _load().mfo_rank_filter(code, x.ctypes.data, n, k, r, y.ctypes.data, arg.ctypes.data,
                                 nthreads)
    if rc != 0:
        raise ValueError(f"mfo_rank_filter returned {rc}")
    return y, arg


def rank_windows(x: np.ndarray, k: int, r: int, starts, nthreads: int = 0):
    """Rank-r elements of the windows x[s .. s+k-1] for each s in ``starts``."""
    x = np.ascontiguousarray(x)
    code = _dtype_code(x)
    starts = np.ascontiguousarray(np.asarray(starts, dtype=np.int64))
    y = np.empty(starts.size, dtype=x.dtype)
    arg = np.empty(starts.size, dtype=np.int64)
    rc = _load().mfo_rank_windows(code, x.ctypes.data, x.size, k, r, starts.ctypes.data,
                                  starts.size, y.ctypes.data, arg.ctypes.data, nthreads)
    if rc != 0:
        raise ValueError(f"mfo_rank_windows returned {rc}")
    return y, arg


def batched(x: np.ndarray, n, k, x_off, y_off, y_total: int, nthreads: int = 0):
    """Filter every packed signal separately; argmed is relative to the signal start."""
    y = np.empty(int(y_total), dtype=x.dtype)
    arg = np.empty(int(y_total), dtype=np.int64)
    for s in range(len(n)):
        xs = x[int(x_off[s]):int(x_off[s]) + int(n[s])]
        ys, a = median_filter(xs, int(k[s]), nthreads=nthreads)
        y[int(y_off[s]):int(y_off[s]) + ys.size] = ys
        arg[int(y_off[s]):int(y_off[s]) + ys.size] = a
    return y, arg


def median_gradient(g: np.ndarray, argmed: np.ndarray, n: int) -> np.ndarray:
    """Gradient of sum_i g[i] * y[i] with respect to x, in float64.

    y[i] equals x[argmed[i]], so dL/dx[j] is the sum of g[i] over the outputs
    whose median element is j (all other partial derivatives are zero where the
    window's values are distinct).
    """
    return np.bincount(np.asarray(argmed, dtype=np.int64),
                       weights=np.asarray(g, dtype=np.float64), minlength=n)
