"""Pins of the oracle's rank filter (order statistic of every window).

The rank-r element of each window under the (value, index) order, for any
k >= 1 (the median of an odd window is r = (k-1)/2, the lower median of an
even window r = k/2 - 1).  Pinned against facts that do not use the oracle's
code: exhaustive brute force over small inputs, the running minimum and
maximum (r = 0 and r = k-1) computed with numpy reductions, monotone inputs
(closed forms), numpy's sort for even-window lower and upper medians, and
IEEE totalOrder on signed zeros.
"""
import itertools

import numpy as np
import pytest

import oracle


def brute(x, k, r):
    ys, args = [], []
    for i in range(x.size - k + 1):
        order = sorted(range(i, i + k), key=lambda j: (x[j], j))
        args.append(order[r])
        ys.append(x[order[r]])
    return np.array(ys, dtype=x.dtype), np.array(args)


def test_exhaustive_small_all_ranks():
    for n in range(1, 7):
        for vals in itertools.product([0, 1, 2], repeat=n):
            x = np.array(vals, dtype=np.int32)
            for k in range(1, n + 1):
                for r in range(k):
                    y, a = oracle.rank_filter(x, k, r)
                    by, ba = brute(x, k, r)
                    assert np.array_equal(y, by) and np.array_equal(a, ba), (vals, k, r)


@pytest.mark.parametrize("k", [1, 2, 5, 8, 33])
def test_min_and_max(k):
    rng = np.random.default_rng(k)
    x = rng.integers(-50, 50, 400).astype(np.int32)         # many ties
    win = np.lib.stride_tricks.sliding_window_view(x, k)
    y0, a0 = oracle.rank_filter(x, k, 0)
    assert np.array_equal(y0, win.min(axis=1))
    assert np.array_equal(a0, np.arange(win.shape[0]) + win.argmin(axis=1))   # first minimum
    y1, a1 = oracle.rank_filter(x, k, k - 1)
    assert np.array_equal(y1, win.max(axis=1))
    last_max = k - 1 - win[:, ::-1].argmax(axis=1)                               # last maximum
    assert np.array_equal(a1, np.arange(win.shape[0]) + last_max)


@pytest.mark.parametrize("k,r", [(4, 1), (4, 2), (10, 0), (10, 4), (10, 9), (7, 6)])
def test_monotone_closed_forms(k, r):
    up = np.arange(100, dtype=np.int32) * 3 - 50
    y, a = oracle.rank_filter(up, k, r)
    assert np.array_equal(a, np.arange(y.size) + r) and np.array_equal(y, up[a])
    down = up[::-1].copy()
    y, a = oracle.rank_filter(down, k, r)
    assert np.array_equal(a, np.arange(y.size) + k - 1 - r)


@pytest.mark.parametrize("k", [2, 4, 6, 10, 64])
def test_even_k_lower_and_upper_median_against_numpy(k):
    rng = np.random.default_rng(100 + k)
    x = rng.random(1000, dtype=np.float32)
    srt = np.sort(np.lib.stride_tricks.sliding_window_view(x, k), axis=1)
    lo, _ = oracle.rank_filter(x, k, k // 2 - 1)
    hi, _ = oracle.rank_filter(x, k, k // 2)
    assert np.array_equal(lo, srt[:, k // 2 - 1])
    assert np.array_equal(hi, srt[:, k // 2])
    # their mean is numpy's (average) median of an even window
    med = np.median(np.lib.stride_tricks.sliding_window_view(x.astype(np.float64), k), axis=1)
    assert np.allclose((lo.astype(np.float64) + hi) / 2, med, rtol=0, atol=0)


def test_signed_zero_total_order():
    x = np.array([0.0, -0.0, 0.0, -0.0], dtype=np.float32)
    y0, a0 = oracle.rank_filter(x, 4, 0)
    y1, a1 = oracle.rank_filter(x, 4, 1)
    y2, a2 = oracle.rank_filter(x, 4, 2)
    assert y0.view(np.uint32)[0] == 0x80000000 and a0[0] == 1
    assert y1.view(np.uint32)[0] == 0x80000000 and a1[0] == 3
    assert y2.view(np.uint32)[0] == 0 and a2[0] == 0


def test_sampled_windows_and_errors():
    x = np.random.default_rng(3).integers(0, 9, 500).astype(np.int32)
    y, a = oracle.rank_filter(x, 6, 2)
    st = np.array([0, 17, 494])
    ys, as_ = oracle.rank_windows(x, 6, 2, st)
    assert np.array_equal(ys, y[st]) and np.array_equal(as_, a[st])
    with pytest.raises(ValueError):
        oracle.rank_filter(x, 6, 6)
    with pytest.raises(ValueError):
        oracle.rank_filter(x, 0, 0)
