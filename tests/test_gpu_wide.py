"""GPU parity for 64-bit elements (int64, float64) on both tiers.

Keys are 64-bit throughout the sort and the joint-rank merges; the
post-processing works on ranks and node ids, unchanged.  Bit-exact y and
exact argmed against the oracle: full comparison where the oracle is quick,
sampled windows across every block-pair boundary otherwise; float64
specials (NaNs, infinities, signed zeros); int64 extremes and ties; the rank
filter; the batched and host-buffer entry points; the entry points that are
32-bit only refuse 64-bit types.
"""
import numpy as np
import pytest
import torch

import oracle
import paper_1406_1717_gb300 as mf
from signals import random_walk_f64, uniform_i64

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


def run(h, x_np, k, rank=None):
    x = torch.from_numpy(np.ascontiguousarray(x_np)).to(DEV)
    m = x_np.size - k + 1
    y = torch.empty(m, dtype=x.dtype, device=DEV)
    a = torch.full((m,), -7, dtype=torch.int32, device=DEV)
    if rank is None:
        mf.mf_filter(h, x, k, y, a)
    else:
        mf.mf_filter_rank(h, x, k, rank, y, a)
    mf.mf_sync(h)
    return y.cpu().numpy(), a.cpu().numpy().astype(np.int64)


def same_bits(a, b):
    return np.array_equal(a.view(np.uint64), b.view(np.uint64))


def signals(n, seed):
    specials = np.array([np.nan, -np.nan, np.inf, -np.inf, 0.0, -0.0, 5e-324, -5e-324,
                         1.7976931348623157e308], dtype=np.float64)
    f = random_walk_f64(n, seed=seed)
    rng = np.random.default_rng(seed)
    idx = rng.integers(0, n, size=max(1, n // 50))
    f[idx] = rng.choice(specials, size=idx.size)
    i = uniform_i64(n, seed=seed)
    i[rng.integers(0, n, size=max(1, n // 20))] = np.iinfo(np.int64).min
    t = (uniform_i64(n, seed=seed + 1) % 9).astype(np.int64)
    return {"float64": f, "int64": i, "int64_ties": t}


@pytest.mark.parametrize("k", [1, 3, 31, 1001, 1025, 4093, 4095])
def test_wide_full(handle, k):
    n = 3 * k + 777
    for name, x in signals(n, k).items():
        y, a = run(handle, x, k)
        ry, ra = oracle.median_filter(x, k)
        assert same_bits(y, ry), (name, k)
        np.testing.assert_array_equal(a, ra, err_msg=name)


@pytest.mark.parametrize("k", [5601, 20001])
def test_wide_large_k_sampled(handle, k):
    n = 4 * k + 99
    for name, x in signals(n, k).items():
        y, a = run(handle, x, k)
        m = n - k + 1
        st = np.unique(np.concatenate([[0, m - 1], np.arange(1, m, k), np.arange(k, m, k),
                                       np.random.default_rng(k).integers(0, m, 100)]))
        ry, ra = oracle.window_medians(x, k, st)
        assert same_bits(y[st], ry), name
        np.testing.assert_array_equal(a[st], ra, err_msg=name)
        idx = np.arange(m)
        assert ((a >= idx) & (a < idx + k)).all() and same_bits(y, x[a])


@pytest.mark.parametrize("k,r", [(4, 1), (64, 31), (1000, 0), (1000, 999)])
def test_wide_rank_filter(handle, k, r):
    x = signals(5 * k + 11, 100 + k)["int64_ties"]
    y, a = run(handle, x, k, r)
    ry, ra = oracle.rank_filter(x, k, r)
    assert same_bits(y, ry)
    np.testing.assert_array_equal(a, ra)


def test_wide_batched_and_host_entry():
    h = mf.mf_create(0, torch.cuda.current_stream(DEV))
    try:
        ks = [31, 255, 1001, 3001, 7001]
        ns = [5000, 20000, 30000, 40000, 50000]
        xs = [random_walk_f64(n, seed=i) for i, n in enumerate(ns)]
        x = np.concatenate(xs)
        x_off = np.cumsum([0] + ns[:-1])
        ms = [n - k + 1 for n, k in zip(ns, ks)]
        y_off = np.cumsum([0] + ms[:-1])
        xd = torch.from_numpy(x).to(DEV)
        y = torch.zeros(sum(ms), dtype=torch.float64, device=DEV)
        mf.mf_filter_batched(h, xd, y, mf.make_segments(ns, ks, x_off, y_off))
        mf.mf_sync(h)
        y_np = y.cpu().numpy()
        for i, (n, k) in enumerate(zip(ns, ks)):
            ry, _ = oracle.median_filter(xs[i], k)
            assert same_bits(y_np[int(y_off[i]):int(y_off[i]) + ms[i]], ry), k
        xh = uniform_i64(33_333, seed=4)
        yh = np.empty(xh.size - 101 + 1, dtype=np.int64)
        ah = np.empty(yh.size, dtype=np.int32)
        mf.mf_filter_host(h, xh, 101, yh, ah)
        ry, ra = oracle.median_filter(xh, 101)
        assert np.array_equal(yh, ry) and np.array_equal(ah.astype(np.int64), ra)
    finally:
        mf.mf_destroy(h)


def test_wide_refused_by_32_bit_entry_points():
    lib = mf.load_library()
    x = torch.zeros(1000, dtype=torch.float64, device=DEV)
    y = torch.zeros(1000, dtype=torch.float64, device=DEV)
    assert lib.mf_filter_noalloc(3, x.data_ptr(), 1000, 11, y.data_ptr(), None, None) == 5
    assert lib.mf_fill_splitmix(2, x.data_ptr(), 1000, 1, None) == 5


def hi_tie_signals(n, seed):
    """64-bit keys whose high 32 bits collide often, so that the order rests
    on the low halves: int64 (a few high words, small low words, negatives)
    and float64 near 1.0 and -2.0 (equal high words, a few ulps apart)."""
    rng = np.random.default_rng(seed)
    i = (rng.integers(-2, 3, size=n).astype(np.int64) << 32) + rng.integers(0, 6, size=n)
    f = np.where(rng.integers(0, 2, size=n) == 0, 1.0, -2.0) * (1.0 + rng.integers(0, 5, size=n) * 2.0 ** -52)
    f[rng.integers(0, n, size=max(1, n // 97))] = np.nan
    return {"int64": i, "float64": f}


@pytest.mark.parametrize("k", [1, 3, 31, 101, 255, 511, 1001, 1021])
def test_wide_sort_variants_on_high_half_ties(k):
    """Merge-sort tiles (two passes over the key halves) and the radix sort
    give the oracle's result, bit for bit, on keys tied in their high half."""
    h = mf.mf_create(0, torch.cuda.current_stream(DEV))
    try:
        n = max(40 * k, 20_000) + 333
        for name, x in hi_tie_signals(n, 7 + k).items():
            ry, ra = oracle.median_filter(x, k)
            for variant in (1, 2):
                mf.mf_set_sort_variant(h, k, variant)
                y, a = run(h, x, k)
                assert same_bits(y, ry), (name, k, variant)
                np.testing.assert_array_equal(a, ra, err_msg=f"{name} variant {variant}")
    finally:
        mf.mf_destroy(h)
