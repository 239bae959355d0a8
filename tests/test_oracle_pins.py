"""Pins of the CPU oracle against facts that do not come from the oracle itself.

Each test checks ``oracle.median_filter`` (the plain per-window sort of
paper Section 1 / Section 2) against something independent of its code:

* brute force over every sequence on {0, 1, 2} up to n = 7 with an order
  statistic computed by counting (no sorting);
* library routines: numpy's median / partition and scipy's median filters;
* closed forms: constant, monotone (y_i = x_{i+h}), k = 1, k = n;
* the paper's lower-bound reduction (Section 2, "Lower Bounds"): a median
  filter over h copies of -inf, a block of h + 1 values, h copies of +inf
  sorts the block -- checked against numpy's sort;
* IEEE 754 totalOrder for float32 (-0 < +0, NaN placement), from a fixture
  listing bit patterns in the standard's order;
* invariance of a single window's median under permutation.

A plausible mistake in the oracle (off-by-one window, wrong rank h, dropped
tie-break, wrong float order, wrong argmed) fails at least one of these.
"""
import itertools
import os

import numpy as np
import pytest
import scipy.ndimage

import oracle
from signals import paper_generator, random_walk_f32, uniform_f32, uniform_i32

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def count_median(window):
    """Order statistic by counting: v with #{< v} <= h < #{<= v} (no sort)."""
    h = (len(window) - 1) // 2
    for v in window:
        less = sum(1 for u in window if u < v)
        leq = sum(1 for u in window if u <= v)
        if less <= h < leq:
            return v
    raise AssertionError("no median found")


def count_argmedian(window, offset):
    """Index (offset + j) of the element with exactly h elements before it in
    the (value, index) order -- counted pairwise, no sort."""
    h = (len(window) - 1) // 2
    for j, v in enumerate(window):
        before = sum(1 for t, u in enumerate(window) if (u, t) < (v, j))
        if before == h:
            return offset + j
    raise AssertionError("no argmedian found")


@pytest.mark.parametrize("n", range(1, 8))
def test_bruteforce_all_ternary_sequences(n):
    for k in range(1, n + 1, 2):
        for seq in itertools.product((0, 1, 2), repeat=n):
            x = np.array(seq, dtype=np.int32)
            y, arg = oracle.median_filter(x, k, nthreads=1)
            assert y.size == n - k + 1
            for i in range(n - k + 1):
                w = list(seq[i:i + k])
                assert y[i] == count_median(w), (seq, k, i)
                assert arg[i] == count_argmedian(w, i), (seq, k, i)


@pytest.mark.parametrize("dtype", ["int32", "float32"])
@pytest.mark.parametrize("k", [1, 3, 5, 31, 101])
def test_matches_scipy_median_filter(dtype, k):
    n = 4000
    x = (uniform_i32(n, seed=7 + k) if dtype == "int32"
         else uniform_f32(n, seed=7 + k))
    y, arg = oracle.median_filter(x, k)
    h = (k - 1) // 2
    ref = scipy.ndimage.median_filter(x, size=k, mode="constant")[h:n - h]
    np.testing.assert_array_equal(y, ref)
    # the argmed element carries the output's bits
    np.testing.assert_array_equal(x[arg], y)


@pytest.mark.parametrize("k", [3, 7, 63])
def test_matches_numpy_median_on_windows(k):
    x = random_walk_f32(3000, seed=11)
    y, _ = oracle.median_filter(x, k)
    win = np.lib.stride_tricks.sliding_window_view(x.astype(np.float64), k)
    np.testing.assert_array_equal(y.astype(np.float64), np.median(win, axis=1))


@pytest.mark.parametrize("gen", ["r-small", "r-block", "r-asc", "r-desc", "r-large"])
def test_paper_generators_match_numpy_partition(gen):
    k = 51
    x = paper_generator(gen, 2500, seed=3)
    y, _ = oracle.median_filter(x, k)
    win = np.lib.stride_tricks.sliding_window_view(x, k)
    ref = np.partition(win, (k - 1) // 2, axis=1)[:, (k - 1) // 2]
    np.testing.assert_array_equal(y, ref)


def test_constant_signal():
    for k in (1, 3, 99):
        x = np.full(500, -17, dtype=np.int32)
        y, arg = oracle.median_filter(x, k)
        assert (y == -17).all()
        # ties are broken by index: rank h of identical values is offset h
        np.testing.assert_array_equal(arg, np.arange(y.size) + (k - 1) // 2)


@pytest.mark.parametrize("gen", ["asc", "desc"])
def test_monotone_signal(gen):
    for k in (3, 11, 201):
        x = paper_generator(gen, 1000, seed=0)
        h = (k - 1) // 2
        y, arg = oracle.median_filter(x, k)
        np.testing.assert_array_equal(y, x[h:h + y.size])
        np.testing.assert_array_equal(arg, np.arange(y.size) + h)


def test_window_one_is_identity():
    x = uniform_f32(777, seed=5)
    y, arg = oracle.median_filter(x, 1)
    np.testing.assert_array_equal(y.view(np.uint32), x.view(np.uint32))
    np.testing.assert_array_equal(arg, np.arange(777))


@pytest.mark.parametrize("n", [1, 3, 9, 1001])
def test_window_equal_to_signal_is_nth_element(n):
    x = uniform_i32(n, seed=n)
    y, arg = oracle.median_filter(x, n)
    h = (n - 1) // 2
    assert y.size == 1
    assert y[0] == np.partition(x, h)[h]
    assert x[arg[0]] == y[0]


def test_single_window_permutation_invariance():
    rng = np.random.default_rng(9)
    base = paper_generator("r-small", 301, seed=2)
    ref, _ = oracle.median_filter(base, 301)
    for _ in range(20):
        y, _ = oracle.median_filter(rng.permutation(base), 301)
        assert y[0] == ref[0]


@pytest.mark.parametrize("h", [1, 2, 7, 50])
def test_lower_bound_reduction_sorts_blocks(h):
    """Paper Section 2: h x (-inf), a block of h + 1 values, h x (+inf); the
    median filter's outputs at offsets 0..h of each unit are the block sorted."""
    rng = np.random.default_rng(h)
    k = 2 * h + 1
    units = 25
    blocks = [rng.integers(-2 ** 30, 2 ** 30, size=h + 1) for _ in range(units)]
    for dtype in ("int32", "float32"):
        lo, hi = ((np.iinfo(np.int32).min, np.iinfo(np.int32).max) if dtype == "int32"
                  else (-np.inf, np.inf))
        parts = []
        for b in blocks:
            vals = b.astype(np.int32) if dtype == "int32" else (b / 7.0).astype(np.float32)
            parts += [np.full(h, lo), vals, np.full(h, hi)]
        x = np.concatenate(parts).astype(dtype)
        y, _ = oracle.median_filter(x, k)
        unit = 3 * h + 1
        for u, b in enumerate(blocks):
            vals = b.astype(np.int32) if dtype == "int32" else (b / 7.0).astype(np.float32)
            np.testing.assert_array_equal(y[u * unit:u * unit + h + 1], np.sort(vals))


def _total_order_fixture():
    vals = []
    with open(os.path.join(GOLDEN, "float32_total_order.txt")) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                vals.append(int(line.split()[0], 16))
    return np.array(vals, dtype=np.uint32)


def test_float32_total_order_fixture():
    """Medians follow IEEE 754 totalOrder on bit patterns (fixture order)."""
    order = _total_order_fixture()
    rng = np.random.default_rng(4)
    for _ in range(300):
        k = int(rng.choice([1, 3, 5, 7, 9, 11, 13]))
        pick = np.sort(rng.choice(order.size, size=k, replace=False))
        expect = order[pick[(k - 1) // 2]]
        x = rng.permutation(order[pick]).view(np.float32)
        y, arg = oracle.median_filter(x, k)
        assert y.view(np.uint32)[0] == expect
        assert x.view(np.uint32)[arg[0]] == expect


def test_signed_zero_is_not_equal_to_positive_zero():
    # -0.0 < +0.0 under totalOrder: the window {-0, +0, +0} has median +0
    x = np.array([0.0, -0.0, 0.0], dtype=np.float32)
    y, _ = oracle.median_filter(x, 3)
    assert y.view(np.uint32)[0] == 0x00000000
    x = np.array([-0.0, 0.0, -0.0], dtype=np.float32)
    y, _ = oracle.median_filter(x, 3)
    assert y.view(np.uint32)[0] == 0x80000000


def test_int32_extremes():
    x = np.array([2 ** 31 - 1, -2 ** 31, 0, 2 ** 31 - 1, -2 ** 31], dtype=np.int32)
    y, _ = oracle.median_filter(x, 5)
    assert y[0] == 0
    y, _ = oracle.median_filter(x, 3)
    np.testing.assert_array_equal(y, [0, 0, 0])


def test_sampled_windows_agree_with_full_filter():
    x = paper_generator("r-block", 5000, seed=8)
    k = 255
    y, arg = oracle.median_filter(x, k)
    starts = np.random.default_rng(1).integers(0, x.size - k + 1, size=300)
    ys, args = oracle.window_medians(x, k, starts)
    np.testing.assert_array_equal(ys, y[starts])
    np.testing.assert_array_equal(args, arg[starts])


def test_rejects_bad_arguments():
    x = np.zeros(10, np.int32)
    for k in (0, 2, 11, -1):
        with pytest.raises(ValueError):
            oracle.median_filter(x, k)


def test_gradient_scatter_matches_finite_differences():
    """Oracle gradient of sum g_i y_i vs central differences in float64."""
    rng = np.random.default_rng(0)
    n, k = 64, 7
    x = rng.permutation(n).astype(np.float64) * 1.0 + rng.normal(0, 0.1, n)
    g = rng.standard_normal(n - k + 1)

    def loss(v):
        win = np.lib.stride_tricks.sliding_window_view(v, k)
        return float(np.dot(np.median(win, axis=1), g))

    _, arg = oracle.median_filter(x.astype(np.float32), k)
    grad = oracle.median_gradient(g, arg, n)
    eps = 1e-4
    fd = np.array([(loss(x + eps * np.eye(n)[j]) - loss(x - eps * np.eye(n)[j])) / (2 * eps)
                   for j in range(n)])
    np.testing.assert_allclose(grad, fd, rtol=1e-6, atol=1e-6)


def test_batched_packing_against_counting():
    """oracle.batched: each packed segment filtered on its own, outputs placed at
    y_off, argmed relative to the segment start -- checked by counting (no sort)
    on small segments of mixed n and k, with gaps between them in x and y."""
    rng = np.random.default_rng(11)
    n = np.array([7, 1, 12, 5, 9])
    k = np.array([3, 1, 5, 5, 1])
    x_off = np.array([0, 9, 12, 30, 40])
    y_total = int((n - k + 1).sum()) + 6
    y_off = np.array([0, 6, 8, 17, 20])
    x = rng.integers(-3, 4, size=60).astype(np.int32)
    y, arg = oracle.batched(x, n, k, x_off, y_off, y_total)
    for s in range(len(n)):
        seg = [int(v) for v in x[x_off[s]:x_off[s] + n[s]]]
        for i in range(n[s] - k[s] + 1):
            w = seg[i:i + k[s]]
            assert y[y_off[s] + i] == count_median(w)
            assert arg[y_off[s] + i] == count_argmedian(w, i)
