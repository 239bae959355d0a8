"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle.

Bar: bit-exact y (raw 32-bit patterns) and exact argmed for every case.
Cases: the workload configurations (small uniform k=31; n=2^26 random walk
and int32 uniform at k=1001, checked on sampled windows including every
pair boundary of sampled pairs), block-boundary sizes n in {k, k+1, 2k-1,
2k, 2k+1, bk, bk+r}, k at tier boundaries, special float values, int32
extremes, heavy ties, the paper's generators, the lower-bound reduction
(checked against numpy's sort, no oracle), host-buffer entry point,
batched entry point and the backward pass.
"""
import numpy as np
import pytest
import torch

import oracle
import paper_1406_1717_gb300 as mf
from signals import (PAPER_GENERATORS, batched_signals, distinct_f32, paper_generator,
                     random_walk_f32, uniform_f32, uniform_i32)

pytestmark = pytest.mark.gpu

DEV = torch.device("cuda:0")


@pytest.fixture(scope="module")
def handle():
    # every window up to the shared-memory pipeline's limit runs on the
    # pipeline here (the large-k tier has tests of its own)
    mf.load_library()
    h = mf.mf_create(0, torch.cuda.current_stream(DEV))
    mf.mf_set_tier_threshold(h, 1 << 30)
    yield h
    mf.mf_destroy(h)


def gpu_filter(h, x_np, k, with_arg=True):
    x = torch.from_numpy(np.ascontiguousarray(x_np)).to(DEV)
    m = x_np.size - k + 1
    y = torch.empty(m, dtype=x.dtype, device=DEV)
    a = torch.full((m,), -7, dtype=torch.int32, device=DEV) if with_arg else None
    mf.mf_filter(h, x, k, y, a)
    mf.mf_sync(h)
    return y.cpu().numpy(), (a.cpu().numpy().astype(np.int64) if with_arg else None)


def assert_bits_equal(got, ref, what=""):
    g, r = got.view(np.uint32), ref.view(np.uint32)
    if not np.array_equal(g, r):
        bad = np.nonzero(g != r)[0]
        raise AssertionError(f"{what}: {bad.size} mismatches, first at {bad[:8]} "
                             f"got {g[bad[:4]]} want {r[bad[:4]]}")


def check_full(h, x, k, what=""):
    y, a = gpu_filter(h, x, k)
    ry, ra = oracle.median_filter(x, k)
    assert_bits_equal(y, ry, what)
    np.testing.assert_array_equal(a, ra, err_msg=what)


# ---------------------------------------------------------------------------
def test_small_uniform_k31_full(handle):
    """n = 100,000 float32 U[0,1), k = 31: every output."""
    check_full(handle, uniform_f32(100_000), 31, "uniform k=31")


@pytest.mark.parametrize("k", [1, 3, 5, 31, 33, 63, 65, 127, 129, 255, 341, 511, 513, 1001, 1021, 1023,
                               1025, 2047, 4093, 4095])
def test_block_boundary_sizes(handle, k):
    rng = np.random.default_rng(k)
    for n in sorted({k, k + 1, 2 * k - 1, 2 * k, 2 * k + 1, 5 * k, 5 * k + int(rng.integers(1, k + 1)),
                     23 * k + 7}):
        if n < k:
            continue
        check_full(handle, random_walk_f32(n, seed=n), k, f"walk n={n} k={k}")
        check_full(handle, uniform_i32(n, seed=n + 1), k, f"int n={n} k={k}")


@pytest.mark.parametrize("gen", PAPER_GENERATORS)
@pytest.mark.parametrize("dtype", ["int32", "float32"])
def test_paper_generators(handle, gen, dtype):
    for k in (7, 101, 1001):
        x = paper_generator(gen, 30_011, seed=k, dtype=dtype)
        check_full(handle, x, k, f"{gen} {dtype} k={k}")


@pytest.mark.parametrize("k", [3, 31, 101, 511, 1001])
def test_ordered_and_unordered_tiles_mixed(handle, k):
    """Sort variant 3 skips tiles whose blocks are all ascending (ties kept in
    position order) or all strictly descending: a signal whose stretches are
    ascending with repeated values, strictly descending, constant, and random
    walk, each several tiles long, checked in full against the oracle with
    that variant and with the default one."""
    rng = np.random.default_rng(k)
    span = 5 * 1024 + 77
    asc = np.sort(rng.integers(0, 50, size=span)).astype(np.float32)          # many ties
    desc = (np.arange(span, 0, -1, dtype=np.float64) * 0.25 - 300.0).astype(np.float32)
    const = np.full(span, 7.0, np.float32)
    x = np.concatenate([asc, desc, random_walk_f32(span, seed=k), const, asc[::-1].copy(),
                        desc[::-1].copy()])
    xi = np.ascontiguousarray(x.astype(np.int32))
    h3 = mf.mf_create(0, torch.cuda.current_stream(DEV))
    try:
        mf.mf_set_sort_variant(h3, k, 3)
        for hh, what in ((h3, "adaptive"), (handle, "default")):
            check_full(hh, x, k, f"ordered mix {what} k={k}")
            check_full(hh, xi, k, f"ordered mix int {what} k={k}")
    finally:
        mf.mf_destroy(h3)


def test_many_tiles_ragged_tail(handle):
    for k in (31, 1001):
        n = 61 * 1001 * 3 + 517
        check_full(handle, random_walk_f32(n, seed=3), k, f"walk tiles k={k}")
        check_full(handle, paper_generator("r-small", n, seed=4), k, f"r-small tiles k={k}")


def test_float_special_values(handle):
    rng = np.random.default_rng(0)
    special = np.array([0x00000000, 0x80000000, 0x7f800000, 0xff800000, 0x7fc00000,
                        0xffc00000, 0x7f800001, 0xff800001, 0x7fffffff, 0xffffffff,
                        0x00000001, 0x80000001, 0x3f800000, 0xbf800000], dtype=np.uint32)
    for k in (3, 31, 255):
        bits = rng.choice(special, size=20_000)
        x = bits.view(np.float32)
        check_full(handle, x, k, f"specials k={k}")
        mix = uniform_f32(20_000, seed=k).view(np.uint32).copy()
        hit = rng.random(20_000) < 0.3
        mix[hit] = rng.choice(special, size=int(hit.sum()))
        check_full(handle, mix.view(np.float32), k, f"mixed specials k={k}")


def test_int32_extremes_and_ties(handle):
    rng = np.random.default_rng(1)
    vals = np.array([-2 ** 31, 2 ** 31 - 1, 0, -1, 1], dtype=np.int32)
    for k in (3, 63, 129, 255, 1001):
        check_full(handle, rng.choice(vals, size=30_000), k, f"int extremes k={k}")
    check_full(handle, np.full(10_000, 5, np.int32), 101, "constant")


@pytest.mark.parametrize("k", [1023, 2047, 3001, 4093, 4095])
def test_long_block_sort_heavy_ties(handle, k):
    """Five distinct values over blocks long enough that the sort splits each
    block into runs and joins them by merging: equal keys must stay in index
    order across the run boundaries (the stable sort of Section 6.1)."""
    rng = np.random.default_rng(k + 11)
    for n in (5 * k + int(rng.integers(1, k)), 9 * k):
        x = rng.integers(-2, 3, size=n).astype(np.int32)
        check_full(handle, x, k, f"5 values n={n} k={k}")
        f = np.where(rng.random(n) < 0.5, np.float32(-0.0), np.float32(0.0))
        f[rng.random(n) < 0.1] = np.float32(1.5)
        check_full(handle, f.astype(np.float32), k, f"signed zeros n={n} k={k}")


def test_impulse_noise_ties(handle):
    b = batched_signals(nseg=8, seed=5)
    for s in range(8):
        x = b.x[b.x_off[s]:b.x_off[s] + b.n[s]]
        check_full(handle, x, int(b.k[s]), f"impulse segment {s}")


@pytest.mark.parametrize("h_", [1, 3, 15, 100, 500])
def test_lower_bound_reduction_sorts(handle, h_):
    """Paper Section 2: -inf x h, block of h+1, +inf x h -> outputs sort the block
    (checked against numpy's sort only)."""
    rng = np.random.default_rng(h_)
    units = 400
    k = 2 * h_ + 1
    blocks = rng.random((units, h_ + 1), dtype=np.float32)
    parts = []
    for b in blocks:
        parts += [np.full(h_, -np.inf, np.float32), b, np.full(h_, np.inf, np.float32)]
    x = np.concatenate(parts)
    y, _ = gpu_filter(handle, x, k, with_arg=False)
    unit = 3 * h_ + 1
    got = np.stack([y[u * unit:u * unit + h_ + 1] for u in range(units)])
    np.testing.assert_array_equal(got, np.sort(blocks, axis=1))


@pytest.mark.parametrize("kind", ["walk_f32", "uniform_i32"])
def test_full_size_k1001_sampled(handle, kind):
    """n = 2^26, k = 1001, the configuration the bench times: the first and the
    last output of every one of the 67,041 block pairs (where a pair's chain
    starts and ends), 10^6 random windows, and both ends of the signal."""
    n, k = 1 << 26, 1001
    x = random_walk_f32(n) if kind == "walk_f32" else uniform_i32(n)
    y, a = gpu_filter(handle, x, k)
    rng = np.random.default_rng(123)
    m = n - k + 1
    pairs = np.arange(1, (n + k - 1) // k)                 # every pair j = 1 .. b-1
    assert pairs.size == 67_041
    starts = np.unique(np.concatenate([(pairs - 1) * k + 1, np.minimum((pairs - 1) * k + k, m - 1),
                                       rng.integers(0, m, size=1_000_000), [0, m - 1]]))
    ry, ra = oracle.window_medians(x, k, starts)
    assert_bits_equal(y[starts], ry, f"{kind} sampled")
    np.testing.assert_array_equal(a[starts], ra)
    # every output is an element of its window (cheap property over all outputs)
    idx = np.arange(m)
    assert ((a >= idx) & (a < idx + k)).all()
    assert_bits_equal(y, x[a], "y == x[argmed]")


def test_max_supported_k_and_unsupported(handle):
    """k up to 2^18 - 1 is served (large k by the global-memory tier); above it
    the call is refused with MF_ERR_UNSUPPORTED before any work."""
    lib = mf.load_library()
    k = (1 << 18) + 1
    xd = torch.zeros(k + 2, device=DEV)
    yd = torch.empty(3, device=DEV)
    assert lib.mf_filter(handle, 1, xd.data_ptr(), k + 2, k, yd.data_ptr(), None) == 8
    k = 16383
    x = uniform_f32(2 * k + 3, seed=k)
    y, a = gpu_filter(handle, x, k)
    ry, ra = oracle.median_filter(x, k)
    assert_bits_equal(y, ry, f"k={k}")
    np.testing.assert_array_equal(a, ra)


def test_argument_errors(handle):
    lib = mf.load_library()
    x = torch.zeros(100, device=DEV)
    y = torch.zeros(100, device=DEV)
    xp, yp = x.data_ptr(), y.data_ptr()
    assert lib.mf_filter(handle, 1, xp, 100, 4, yp, None) == 3       # even k
    assert lib.mf_filter(handle, 1, xp, 100, 101, yp, None) == 4     # k > n
    assert lib.mf_filter(handle, 1, xp, 100, 0, yp, None) == 4       # k < 1
    assert lib.mf_filter(handle, 1, xp, 0, 1, yp, None) == 2         # n < 1
    assert lib.mf_filter(handle, 7, xp, 100, 3, yp, None) == 5       # dtype
    assert lib.mf_filter(handle, 1, xp, 100, 3, xp + 8, None) == 9   # overlap
    assert lib.mf_filter(handle, 1, None, 100, 3, yp, None) == 1     # null


def test_host_entry_point_matches_device(handle):
    x = random_walk_f32(300_007, seed=9)
    k = 1001
    y = np.empty(x.size - k + 1, np.float32)
    a = np.empty(x.size - k + 1, np.int32)
    mf.mf_filter_host(handle, x, k, y, a)
    yd, ad = gpu_filter(handle, x, k)
    assert_bits_equal(y, yd, "host vs device")
    np.testing.assert_array_equal(a.astype(np.int64), ad)


def test_batched_matches_oracle(handle):
    b = batched_signals(nseg=64, seed=11, n_hi=20_000)
    x = torch.from_numpy(b.x).to(DEV)
    y = torch.empty(b.y_total, device=DEV)
    a = torch.empty(b.y_total, dtype=torch.int32, device=DEV)
    segs = mf.make_segments(b.n, b.k, b.x_off, b.y_off)
    mf.mf_filter_batched(handle, x, y, segs, a)
    mf.mf_sync(handle)
    ry, ra = oracle.batched(b.x, b.n, b.k, b.x_off, b.y_off, b.y_total)
    assert_bits_equal(y.cpu().numpy(), ry, "batched")
    np.testing.assert_array_equal(a.cpu().numpy().astype(np.int64), ra)


def test_backward_matches_oracle_gradient(handle):
    n, k = 65_536, 63
    x_np = distinct_f32(n, seed=2)
    g_np = np.random.default_rng(3).standard_normal(n - k + 1).astype(np.float32)
    _, a = gpu_filter(handle, x_np, k)
    gy = torch.from_numpy(g_np).to(DEV)
    ad = torch.from_numpy(a.astype(np.int32)).to(DEV)
    gx = torch.empty(n, device=DEV)
    mf.mf_filter_backward(handle, gy, ad, n, k, gx)
    mf.mf_sync(handle)
    _, ra = oracle.median_filter(x_np, k)
    ref = oracle.median_gradient(g_np.astype(np.float64), ra, n)
    # each gx[j] sums at most k float32 terms: bound the rounding by k * eps * sum|g|
    absref = oracle.median_gradient(np.abs(g_np).astype(np.float64), ra, n)
    np.testing.assert_array_less(np.abs(gx.cpu().numpy() - ref), k * 6e-8 * absref + 1e-30)


def test_backward_rows_equals_rows_one_by_one(handle):
    """One launch over equal rows gives each row's single-row result, bit for bit."""
    rng = np.random.default_rng(4)
    for rows, n, k in ((5, 3001, 31), (3, 1000, 1), (2, 700, 699)):
        m = n - k + 1
        a = np.stack([np.minimum(np.arange(m) + rng.integers(0, k, m), n - 1) for _ in range(rows)])
        g = rng.standard_normal((rows, m)).astype(np.float32)
        ad = torch.from_numpy(a.astype(np.int32)).to(DEV)
        gy = torch.from_numpy(g).to(DEV)
        gx = torch.full((rows, n), np.nan, device=DEV)
        mf.mf_filter_backward_rows(handle, gy, ad, rows, n, k, gx)
        one = torch.full((rows, n), np.nan, device=DEV)
        for r in range(rows):
            mf.mf_filter_backward(handle, gy[r], ad[r], n, k, one[r])
        mf.mf_sync(handle)
        assert np.array_equal(gx.cpu().numpy().view(np.uint32), one.cpu().numpy().view(np.uint32))
        ref = np.stack([oracle.median_gradient(g[r].astype(np.float64), a[r], n) for r in range(rows)])
        bound = np.stack([oracle.median_gradient(np.abs(g[r]).astype(np.float64), a[r], n) for r in range(rows)])
        assert np.all(np.abs(gx.cpu().numpy() - ref) <= k * 6e-8 * bound + 1e-30)


@pytest.mark.parametrize("n,k,kind", [(5_000_000, 1001, "walk"), (3_000_011, 20001, "int"),
                                      (2_500_000, 31, "walk64")])
def test_host_entry_point_chunked(handle, n, k, kind):
    """Signals above 2^20 outputs go through the host entry point in chunks on
    two streams; the result (and argmed, shifted per chunk) equals one device call."""
    from signals import random_walk_f64
    x = {"walk": lambda: random_walk_f32(n, seed=n),
         "int": lambda: uniform_i32(n, seed=n),
         "walk64": lambda: random_walk_f64(n, seed=n)}[kind]()
    y = np.empty(n - k + 1, x.dtype)
    a = np.empty(n - k + 1, np.int32)
    mf.mf_filter_host(handle, x, k, y, a)
    xd = torch.from_numpy(x).to(DEV)
    yd = torch.empty(n - k + 1, dtype=xd.dtype, device=DEV)
    ad = torch.empty(n - k + 1, dtype=torch.int32, device=DEV)
    mf.mf_filter(handle, xd, k, yd, ad)
    mf.mf_sync(handle)
    assert np.array_equal(y.view(np.uint8), yd.cpu().numpy().view(np.uint8))
    np.testing.assert_array_equal(a, ad.cpu().numpy())
    st = np.random.default_rng(1).integers(0, n - k + 1, 200)
    ry, ra = oracle.window_medians(x, k, st)
    assert np.array_equal(y[st].view(np.uint8), ry.view(np.uint8))
    np.testing.assert_array_equal(a[st].astype(np.int64), ra)
