"""mf_filter_noalloc: the median filter for callers that cannot allocate
device memory (for example programs whose device memory comes only from their
own pool, or real-time loops that cannot wait for an allocation).

It runs the same kernels as mf_filter but keeps their scratch in a fixed
array inside the library instead of a workspace it allocates.  This test
calls it through the C ABI several times in a row, on different inputs and
window sizes, and checks each result bit for bit against mf_filter: the fused
path (k = 1001, k = 31) and, right after them on the scratch they left, the
four-kernel path (k = 2047).  It also checks the size limit: the largest
accepted n at k = 1001 runs and matches, one sample more is refused.  The
file sorts last so that a run stopping at the first failure has already run
every other test.
"""
import ctypes

import numpy as np
import pytest
import torch

import paper_1406_1717_gb300 as mf
from signals import random_walk_f32, uniform_i32

pytestmark = pytest.mark.gpu

DEV = torch.device("cuda:0")


def _reference(x, k):
    h = mf.mf_create(0, torch.cuda.current_stream(DEV))
    try:
        y = torch.empty(x.numel() - k + 1, dtype=x.dtype, device=DEV)
        a = torch.empty(x.numel() - k + 1, dtype=torch.int32, device=DEV)
        mf.mf_filter(h, x, k, y, a)
        mf.mf_sync(h)
    finally:
        mf.mf_destroy(h)
    return y.cpu().numpy(), a.cpu().numpy()


def test_noalloc_matches_mf_filter_on_two_calls_in_a_row():
    lib = mf.load_library()
    stream = torch.cuda.current_stream(DEV)
    cases = [(random_walk_f32(700_001, seed=41), 1001, 1),
             (uniform_i32(300_007, seed=42), 31, 0),
             (random_walk_f32(600_011, seed=43), 2047, 1)]
    outs = []
    for x_np, k, code in cases:
        x = torch.from_numpy(x_np).to(DEV)
        m = x_np.size - k + 1
        y = torch.full((m,), -1, dtype=x.dtype, device=DEV)
        a = torch.full((m,), -1, dtype=torch.int32, device=DEV)
        st = lib.mf_filter_noalloc(code, ctypes.c_void_p(x.data_ptr()), x_np.size, k,
                                   ctypes.c_void_p(y.data_ptr()), ctypes.c_void_p(a.data_ptr()),
                                   ctypes.c_void_p(stream.cuda_stream))
        assert st == 0, mf.mf_status_str(st)
        torch.cuda.synchronize(DEV)
        outs.append((x, k, y.cpu().numpy(), a.cpu().numpy()))
    for x, k, y, a in outs:
        ry, ra = _reference(x, k)
        np.testing.assert_array_equal(y.view(np.uint32), ry.view(np.uint32))
        np.testing.assert_array_equal(a, ra)


def test_noalloc_refuses_requests_beyond_its_scratch():
    lib = mf.load_library()
    n, k = 4_000_000, 1001
    x = torch.zeros(n, dtype=torch.float32, device=DEV)
    y = torch.zeros(n - k + 1, dtype=torch.float32, device=DEV)
    st = lib.mf_filter_noalloc(1, ctypes.c_void_p(x.data_ptr()), n, k,
                               ctypes.c_void_p(y.data_ptr()), None, None)
    assert st == 12                       # MF_ERR_TOO_LARGE, nothing launched
    assert "TOO_LARGE" in mf.mf_status_str(st)


def test_noalloc_size_limit_at_k1001():
    """At k = 1001 the 32 MiB array holds the scratch of n = 1,850,849 samples
    (the larger of 12 kp bytes per block + 6 kp per pair and 8 kw + 2 kp per
    pair, kp = 1008, kw = 1008): that n runs and matches mf_filter, one sample
    more (a new block) is refused."""
    lib = mf.load_library()
    k, n_max = 1001, 1_850_849
    stream = torch.cuda.current_stream(DEV)
    x_np = uniform_i32(n_max + 1, seed=44)
    x = torch.from_numpy(x_np).to(DEV)
    y = torch.full((n_max + 1 - k + 1,), -1, dtype=x.dtype, device=DEV)
    st = lib.mf_filter_noalloc(0, ctypes.c_void_p(x.data_ptr()), n_max + 1, k,
                               ctypes.c_void_p(y.data_ptr()), None, ctypes.c_void_p(stream.cuda_stream))
    assert st == 12
    st = lib.mf_filter_noalloc(0, ctypes.c_void_p(x.data_ptr()), n_max, k,
                               ctypes.c_void_p(y.data_ptr()), None, ctypes.c_void_p(stream.cuda_stream))
    assert st == 0, mf.mf_status_str(st)
    torch.cuda.synchronize(DEV)
    ry, _ = _reference(x[:n_max], k)
    got = y[:n_max - k + 1].cpu().numpy()
    np.testing.assert_array_equal(got.view(np.uint32), ry.view(np.uint32))
