"""GPU parity of the large-k tier (global-memory merge tiers and segmented
dancing-links chains) for window sizes above the shared-memory pipeline.

Bar: bit-exact y and exact argmed against the CPU oracle.  Full comparison
where the oracle finishes in seconds; otherwise sampled windows that include
every block-pair boundary and every chain-segment boundary, plus properties
checked on all outputs (argmed inside its window, y == x[argmed]).
Cases: k just above the pipeline limit, k of the serving configuration's
range (up to 100,001), float32 random walk and uniform, int32 uniform over
[0, 65536) (many ties at large k), ragged last blocks, n = k, n = 2k and
block-boundary sizes, the batched entry point mixing both tiers, and the
host-buffer entry point.
"""
import numpy as np
import pytest
import torch

import oracle
import paper_1406_1717_gb300 as mf
from signals import random_walk_f32, uniform_f32, uniform_i32

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")


@pytest.fixture(scope="module")
def handle():
    mf.load_library()
    h = mf.mf_create(0, torch.cuda.current_stream(DEV))
    yield h
    mf.mf_destroy(h)


def gpu_filter(h, x_np, k):
    x = torch.from_numpy(np.ascontiguousarray(x_np)).to(DEV)
    m = x_np.size - k + 1
    y = torch.empty(m, dtype=x.dtype, device=DEV)
    a = torch.full((m,), -7, dtype=torch.int32, device=DEV)
    mf.mf_filter(h, x, k, y, a)
    mf.mf_sync(h)
    return y.cpu().numpy(), a.cpu().numpy().astype(np.int64)


def bits(v):
    return v.view(np.uint32)


def segment_starts(n, k, rng, extra=400):
    """Windows around every pair boundary and every chain-segment boundary."""
    m = n - k + 1
    seg = max(1, min(32, -(-k // 1024)))
    L = -(-k // seg)
    s = {0, m - 1}
    for q in range(-(-n // k)):
        for t in range(seg + 1):
            o = 1 + q * k + t * L
            for d in (-1, 0, 1):
                if 0 <= o + d < m:
                    s.add(o + d)
    s.update(rng.integers(0, m, size=extra).tolist())
    return np.array(sorted(s), dtype=np.int64)


def check(h, x, k, full=False, seed=0):
    y, a = gpu_filter(h, x, k)
    m = x.size - k + 1
    idx = np.arange(m)
    assert ((a >= idx) & (a < idx + k)).all()
    assert np.array_equal(bits(y), bits(x[a]))
    if full:
        ry, ra = oracle.median_filter(x, k)
        assert np.array_equal(bits(y), bits(ry))
        np.testing.assert_array_equal(a, ra)
    else:
        st = segment_starts(x.size, k, np.random.default_rng(seed))
        ry, ra = oracle.window_medians(x, k, st)
        assert np.array_equal(bits(y[st]), bits(ry))
        np.testing.assert_array_equal(a[st], ra)


@pytest.mark.parametrize("k", [9345, 10001])
@pytest.mark.parametrize("kind", ["walk", "i32", "uniform"])
def test_just_above_pipeline_full(handle, k, kind):
    n = 3 * k + 1234
    x = {"walk": random_walk_f32, "i32": lambda n, seed: uniform_i32(n, seed=seed) % 65536,
         "uniform": uniform_f32}[kind](n, seed=k)
    check(handle, np.ascontiguousarray(x), k, full=True)


@pytest.mark.parametrize("n_of_k", [lambda k: k, lambda k: k + 1, lambda k: 2 * k - 1,
                                    lambda k: 2 * k, lambda k: 2 * k + 1])
def test_block_boundary_sizes(handle, n_of_k):
    k = 12001
    x = uniform_f32(n_of_k(k), seed=5)
    check(handle, x, k, full=True)


@pytest.mark.parametrize("k", [20001, 49999, 100001])
def test_serving_range_sampled(handle, k):
    n = 5 * k + 777
    check(handle, random_walk_f32(n, seed=k), k, seed=k)
    xi = np.ascontiguousarray(uniform_i32(n, seed=k + 1) % 65536).astype(np.int32)
    check(handle, xi, k, seed=k + 1)


def test_maximum_k(handle):
    k = (1 << 18) - 1
    x = uniform_f32(2 * k + 4321, seed=11)
    check(handle, x, k, seed=11)


def test_large_k_ten_million_sampled(handle):
    n, k = 10_000_000, 100_001
    x = uniform_f32(n, seed=77)
    check(handle, x, k, seed=77)


def test_batched_mixes_both_tiers(handle):
    rng = np.random.default_rng(3)
    ks = [31, 12001, 1001, 30001, 8005, 4095]
    ns = [5000, 40000, 70000, 95000, 30000, 20000]
    xs = [uniform_f32(n, seed=100 + i) for i, n in enumerate(ns)]
    x = np.concatenate(xs)
    x_off = np.cumsum([0] + ns[:-1])
    ms = [n - k + 1 for n, k in zip(ns, ks)]
    y_off = np.cumsum([0] + ms[:-1])
    xd = torch.from_numpy(x).to(DEV)
    y = torch.full((sum(ms),), -1.0, device=DEV)
    a = torch.full((sum(ms),), -1, dtype=torch.int32, device=DEV)
    mf.mf_filter_batched(handle, xd, y, mf.make_segments(ns, ks, x_off, y_off), a)
    mf.mf_sync(handle)
    y_np, a_np = y.cpu().numpy(), a.cpu().numpy().astype(np.int64)
    for i, (n, k) in enumerate(zip(ns, ks)):
        sl = slice(int(y_off[i]), int(y_off[i]) + ms[i])
        ys, as_ = gpu_filter(handle, xs[i], k)
        assert np.array_equal(bits(y_np[sl]), bits(ys)), i
        np.testing.assert_array_equal(a_np[sl], as_)
        st = np.unique(np.concatenate([rng.integers(0, ms[i], 300), [0, ms[i] - 1]]))
        ry, ra = oracle.window_medians(xs[i], k, st)
        assert np.array_equal(bits(y_np[sl][st]), bits(ry)), i
        np.testing.assert_array_equal(a_np[sl][st], ra)
    del rng


def test_host_entry_point_large_k(handle):
    k = 25001
    x = random_walk_f32(4 * k + 99, seed=4)
    y = np.empty(x.size - k + 1, np.float32)
    a = np.empty(x.size - k + 1, np.int32)
    mf.mf_filter_host(handle, x, k, y, a)
    yd, ad = gpu_filter(handle, x, k)
    assert np.array_equal(bits(y), bits(yd))
    np.testing.assert_array_equal(a.astype(np.int64), ad)


@pytest.fixture(scope="module")
def large_handle():
    """A handle that sends every window size to the large-k tier."""
    mf.load_library()
    h = mf.mf_create(0, torch.cuda.current_stream(DEV))
    mf.mf_set_tier_threshold(h, 1)
    yield h
    mf.mf_destroy(h)


@pytest.mark.parametrize("k", [1, 3, 31, 101, 1001, 1025, 4095])
@pytest.mark.parametrize("kind", ["walk", "i32_ties", "uniform"])
def test_large_tier_at_small_k_full(large_handle, k, kind):
    n = max(5 * k + 13, 3001)
    x = {"walk": lambda: random_walk_f32(n, seed=k),
         "i32_ties": lambda: (uniform_i32(n, seed=k) % 7).astype(np.int32),
         "uniform": lambda: uniform_f32(n, seed=k)}[kind]()
    check(large_handle, np.ascontiguousarray(x), k, full=True)


def test_tiers_agree_and_threshold_resets(handle, large_handle):
    x = random_walk_f32(300_001, seed=12)
    for k in (2047, 9343):
        y1, a1 = gpu_filter(handle, x, k)
        y2, a2 = gpu_filter(large_handle, x, k)
        assert np.array_equal(bits(y1), bits(y2))
        np.testing.assert_array_equal(a1, a2)
    h = mf.mf_create(0, torch.cuda.current_stream(DEV))
    try:
        mf.mf_set_tier_threshold(h, 101)
        mf.mf_set_tier_threshold(h, 0)
        l0 = mf.mf_launch_count(h)
        gpu_filter(h, x, 1001)
        assert mf.mf_launch_count(h) - l0 == 3          # fused sort, chains, store
        l0 = mf.mf_launch_count(h)
        gpu_filter(h, x, 2047)
        assert mf.mf_launch_count(h) - l0 == 4          # the four-kernel pipeline
        l0 = mf.mf_launch_count(h)
        gpu_filter(h, x, 6001)                           # default crossover: large-k tier
        assert mf.mf_launch_count(h) - l0 > 4
    finally:
        mf.mf_destroy(h)


def _batch(ns, ks, dtype, seed):
    gen = uniform_i32 if dtype == "int32" else random_walk_f32
    xs = [gen(n, seed=seed + i) for i, n in enumerate(ns)]
    if dtype == "int32":
        xs = [(v % 65536).astype(np.int32) for v in xs]        # many ties at large k
    x_off = np.cumsum([0] + list(ns[:-1]))
    ms = [n - k + 1 for n, k in zip(ns, ks)]
    y_off = np.cumsum([0] + ms[:-1])
    return xs, np.concatenate(xs), x_off, y_off, ms


@pytest.mark.parametrize("dtype", ["float32", "int32"])
def test_batched_large_signals_share_one_launch_sequence(handle, dtype):
    """The large-k signals of a batch run in one launch sequence of the
    global-memory tier: a batch with five of them (ragged, n = k, n = 2k + 1)
    makes as many launches as one with a single one of the same largest k,
    and every output equals the signal filtered alone (bit for bit, with
    argmed)."""
    small_n, small_k = [4000, 9000, 30000], [31, 255, 1001]
    one = (small_n + [60_000], small_k + [20_001])
    five = (small_n + [60_000, 9_345, 2 * 12_001 + 1, 41_003, 80_000],
            small_k + [20_001, 9_345, 12_001, 16_385, 15_001])
    counts = []
    for ns, ks in (one, five):
        xs, x, x_off, y_off, ms = _batch(ns, ks, dtype, seed=70)
        xd = torch.from_numpy(x).to(DEV)
        y = torch.full((sum(ms),), -1, dtype=xd.dtype, device=DEV)
        a = torch.full((sum(ms),), -1, dtype=torch.int32, device=DEV)
        segs = mf.make_segments(ns, ks, x_off, y_off)
        mf.mf_filter_batched(handle, xd, y, segs, a)          # sizes the workspace
        mf.mf_sync(handle)
        l0 = mf.mf_launch_count(handle)
        mf.mf_filter_batched(handle, xd, y, segs, a)
        mf.mf_sync(handle)
        counts.append(mf.mf_launch_count(handle) - l0)
        y_np, a_np = y.cpu().numpy(), a.cpu().numpy().astype(np.int64)
        for i, (n, k) in enumerate(zip(ns, ks)):
            sl = slice(int(y_off[i]), int(y_off[i]) + ms[i])
            ys, as_ = gpu_filter(handle, xs[i], k)
            assert np.array_equal(bits(y_np[sl]), bits(ys)), (dtype, n, k)
            assert np.array_equal(a_np[sl], as_), (dtype, n, k)
    assert counts[0] == counts[1], counts


def test_batched_large_signals_against_oracle(handle):
    """Three large-k signals in one batched call, sampled windows (every pair
    and chain-segment boundary) against the oracle."""
    rng = np.random.default_rng(11)
    ns, ks = [50_000, 30_001, 70_003], [10_001, 15_001, 30_001]
    xs, x, x_off, y_off, ms = _batch(ns, ks, "float32", seed=90)
    xd = torch.from_numpy(x).to(DEV)
    y = torch.full((sum(ms),), -1.0, device=DEV)
    a = torch.full((sum(ms),), -1, dtype=torch.int32, device=DEV)
    mf.mf_filter_batched(handle, xd, y, mf.make_segments(ns, ks, x_off, y_off), a)
    mf.mf_sync(handle)
    y_np, a_np = y.cpu().numpy(), a.cpu().numpy().astype(np.int64)
    for i, (n, k) in enumerate(zip(ns, ks)):
        starts = segment_starts(n, k, rng)
        ry, ra = oracle.window_medians(xs[i], k, starts)
        sl = y_np[int(y_off[i]):int(y_off[i]) + ms[i]]
        al = a_np[int(y_off[i]):int(y_off[i]) + ms[i]]
        assert np.array_equal(bits(sl[starts]), bits(ry)), (n, k)
        assert np.array_equal(al[starts], ra), (n, k)
