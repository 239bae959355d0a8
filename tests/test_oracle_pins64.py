"""Pins of the oracle for 64-bit elements (int64, float64).

The same definition as for 32-bit elements: the element of rank r in each
window under (value, index) order, values compared as signed integers or by
IEEE 754 totalOrder.  Pinned against brute force with Python integers,
scipy.ndimage.median_filter and numpy's sort on float64, a float64
totalOrder fixture (tests/golden/float64_total_order.txt, IEEE 754-2008
Section 5.10), int64 extremes and signed zeros.
"""
import itertools
import os

import numpy as np
import pytest

import oracle
from signals import random_walk_f64, uniform_i64

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "float64_total_order.txt")


def brute(vals, k, r):
    out, arg = [], []
    for i in range(len(vals) - k + 1):
        order = sorted(range(i, i + k), key=lambda j: (vals[j], j))
        out.append(vals[order[r]])
        arg.append(order[r])
    return out, arg


def test_int64_brute_force_with_extremes():
    big = [-2 ** 63, -2 ** 62 - 3, -1, 0, 1, 2 ** 40, 2 ** 63 - 1]
    rng = np.random.default_rng(2)
    for _ in range(200):
        n = int(rng.integers(1, 12))
        vals = [int(v) for v in rng.choice(big, size=n)]
        x = np.array(vals, dtype=np.int64)
        k = int(rng.integers(1, n + 1))
        r = int(rng.integers(0, k))
        y, a = oracle.rank_filter(x, k, r)
        by, ba = brute(vals, k, r)
        assert [int(v) for v in y] == by and list(a) == ba
    for vals in itertools.product([-2 ** 63, 0, 2 ** 63 - 1], repeat=5):
        x = np.array(vals, dtype=np.int64)
        y, a = oracle.median_filter(x, 3)
        by, ba = brute(list(vals), 3, 1)
        assert [int(v) for v in y] == by and list(a) == ba


def test_float64_against_scipy_and_numpy():
    scipy_ndimage = pytest.importorskip("scipy.ndimage")
    x = random_walk_f64(5000, seed=3)
    for k in (1, 3, 31, 101):
        y, _ = oracle.median_filter(x, k)
        h = (k - 1) // 2
        ref = scipy_ndimage.median_filter(x, size=k, mode="nearest")[h:x.size - h]
        np.testing.assert_array_equal(y, ref)
    srt = np.sort(np.lib.stride_tricks.sliding_window_view(x, 10), axis=1)
    for r in (0, 4, 5, 9):
        y, _ = oracle.rank_filter(x, 10, r)
        np.testing.assert_array_equal(y, srt[:, r])


def test_float64_total_order_fixture():
    order = np.array([int(l.split()[0], 16) for l in open(GOLDEN)
                      if l.strip() and not l.startswith("#")], dtype=np.uint64)
    rng = np.random.default_rng(5)
    for _ in range(300):
        k = int(rng.choice([1, 2, 3, 5, 8, 13]))
        pick = np.sort(rng.choice(order.size, size=k, replace=False))
        r = int(rng.integers(0, k))
        x = rng.permutation(order[pick]).view(np.float64)
        y, a = oracle.rank_filter(x, k, r)
        assert y.view(np.uint64)[0] == order[pick[r]]
        assert x.view(np.uint64)[a[0]] == order[pick[r]]


def test_int64_uniform_sampled_windows_match_numpy():
    x = uniform_i64(3000, seed=7)
    k = 255
    y, a = oracle.median_filter(x, k)
    srt = np.sort(np.lib.stride_tricks.sliding_window_view(x, k), axis=1)
    np.testing.assert_array_equal(y, srt[:, (k - 1) // 2])
    assert np.array_equal(y, x[a])
    st = np.array([0, 99, 2745])
    ys, as_ = oracle.window_medians(x, k, st)
    assert np.array_equal(ys, y[st]) and np.array_equal(as_, a[st])
