"""GPU parity of the rank filter (mf_filter_rank): any window size k >= 1,
any 0-based rank r < k, on both tiers (shared-memory pipeline and large-k),
against the oracle's rank filter.  Even k with r = k/2 - 1 is the lower
median.  Bit-exact y and exact argmed."""
import numpy as np
import pytest
import torch

import oracle
import paper_1406_1717_gb300 as mf
from signals import random_walk_f32, uniform_f32, uniform_i32

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")


@pytest.fixture(scope="module", params=["default", "large"])
def handle(request):
    mf.load_library()
    h = mf.mf_create(0, torch.cuda.current_stream(DEV))
    if request.param == "large":
        mf.mf_set_tier_threshold(h, 1)
    yield h
    mf.mf_destroy(h)


def run(h, x_np, k, r):
    x = torch.from_numpy(np.ascontiguousarray(x_np)).to(DEV)
    m = x_np.size - k + 1
    y = torch.empty(m, dtype=x.dtype, device=DEV)
    a = torch.full((m,), -7, dtype=torch.int32, device=DEV)
    mf.mf_filter_rank(h, x, k, r, y, a)
    mf.mf_sync(h)
    return y.cpu().numpy(), a.cpu().numpy().astype(np.int64)


def ranks_of(k):
    return sorted({0, 1 % k, max(0, k // 2 - 1), k // 2 if k > 1 else 0, (k - 1) // 2,
                   max(0, k - 2), k - 1})


@pytest.mark.parametrize("k", [1, 2, 3, 4, 31, 32, 64, 100, 1000, 1022, 2048])
def test_rank_filter_full(handle, k):
    n = 3 * k + 777
    xs = [random_walk_f32(n, seed=k), (uniform_i32(n, seed=k) % 5).astype(np.int32)]
    for x in xs:
        for r in ranks_of(k):
            y, a = run(handle, x, k, r)
            ry, ra = oracle.rank_filter(x, k, r)
            assert np.array_equal(y.view(np.uint32), ry.view(np.uint32)), (k, r, x.dtype)
            np.testing.assert_array_equal(a, ra)


@pytest.mark.parametrize("k", [6000, 20000])
def test_even_large_k_lower_median_sampled(handle, k):
    n = 4 * k + 321
    x = uniform_f32(n, seed=k)
    r = k // 2 - 1
    y, a = run(handle, x, k, r)
    m = n - k + 1
    rng = np.random.default_rng(k)
    st = np.unique(np.concatenate([[0, m - 1], rng.integers(0, m, 150),
                                   np.arange(1, m, k), np.arange(k, m, k)]))
    ry, ra = oracle.rank_windows(x, k, r, st)
    assert np.array_equal(y[st].view(np.uint32), ry.view(np.uint32))
    np.testing.assert_array_equal(a[st], ra)
    idx = np.arange(m)
    assert ((a >= idx) & (a < idx + k)).all() and np.array_equal(y.view(np.uint32), x[a].view(np.uint32))


def test_rank_arguments(handle):
    lib = mf.load_library()
    x = torch.zeros(100, device=DEV)
    y = torch.zeros(100, device=DEV)
    assert lib.mf_filter_rank(handle, 1, x.data_ptr(), 100, 4, 4, y.data_ptr(), None) == 13
    assert lib.mf_filter_rank(handle, 1, x.data_ptr(), 100, 4, -1, y.data_ptr(), None) == 13
    assert lib.mf_filter_rank(handle, 1, x.data_ptr(), 100, 101, 0, y.data_ptr(), None) == 4
    assert lib.mf_filter(handle, 1, x.data_ptr(), 100, 4, y.data_ptr(), None) == 3   # even k: median needs odd
    assert lib.mf_filter_rank(handle, 1, x.data_ptr(), 100, 4, 1, y.data_ptr(), None) == 0
    mf.mf_sync(handle)
