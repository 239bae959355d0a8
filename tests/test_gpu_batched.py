"""Batched filtering: many signals of different n and k in one call.

* the batched configuration (4096 float32 signals, n log-uniform in
  [1000, 262144], odd k log-uniform in [3, 4095], 10 % +-1e3 impulses) is
  bit-exact against filtering each signal alone with mf_filter, and against
  the oracle on a sample of signals;
* the call launches a bounded number of kernels, independent of the count;
* the batched call captured into a CUDA graph and replayed gives the same
  result; a later uncaptured call does not disturb the graph.
"""
import numpy as np
import pytest
import torch

import oracle
import paper_1406_1717_gb300 as mf
from signals import batched_signals

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")


@pytest.fixture(scope="module")
def batch():
    return batched_signals(nseg=4096, seed=20140607)


def _run_batched(h, b, x, with_arg=True):
    y = torch.full((b.y_total,), -1.0, device=DEV)
    a = torch.full((b.y_total,), -1, dtype=torch.int32, device=DEV) if with_arg else None
    mf.mf_filter_batched(h, x, y, mf.make_segments(b.n, b.k, b.x_off, b.y_off), a)
    return y, a


def test_batched_configuration_matches_single_calls(batch):
    b = batch
    h = mf.mf_create(0, torch.cuda.current_stream(DEV))
    try:
        x = torch.from_numpy(b.x).to(DEV)
        l0 = mf.mf_launch_count(h)
        y, a = _run_batched(h, b, x)
        mf.mf_sync(h)
        # at most four pipeline kernels for each of six window classes, plus
        # one launch sequence of the large-k tier for the signals at or above
        # the tier threshold: six kernels and ceil(log2(kmax / 1024)) merge tiers
        kmax = int(b.k.max())
        tiers = max(0, int(np.ceil(np.log2(max(1.0, kmax / 1024)))))
        assert mf.mf_launch_count(h) - l0 <= 24 + 6 + tiers
        y_np, a_np = y.cpu().numpy(), a.cpu().numpy()
        for s in range(len(b.n)):
            n, k = int(b.n[s]), int(b.k[s])
            xs = x[int(b.x_off[s]):int(b.x_off[s]) + n]
            ys = torch.empty(n - k + 1, device=DEV)
            as_ = torch.empty(n - k + 1, dtype=torch.int32, device=DEV)
            mf.mf_filter(h, xs, k, ys, as_)
            sl = slice(int(b.y_off[s]), int(b.y_off[s]) + n - k + 1)
            assert np.array_equal(y_np[sl].view(np.uint32), ys.cpu().numpy().view(np.uint32)), s
            assert np.array_equal(a_np[sl], as_.cpu().numpy()), s
        for s in range(0, len(b.n), 97):
            n, k = int(b.n[s]), int(b.k[s])
            xs = b.x[int(b.x_off[s]):int(b.x_off[s]) + n]
            ry, ra = oracle.median_filter(xs, k)
            sl = slice(int(b.y_off[s]), int(b.y_off[s]) + n - k + 1)
            np.testing.assert_array_equal(y_np[sl].view(np.uint32), ry.view(np.uint32))
            np.testing.assert_array_equal(a_np[sl].astype(np.int64), ra)
    finally:
        mf.mf_destroy(h)


def test_batched_cuda_graph_capture_and_replay():
    b = batched_signals(nseg=256, seed=3, n_hi=50_000)
    stream = torch.cuda.Stream(DEV)
    h = mf.mf_create(0, stream)
    try:
        x = torch.from_numpy(b.x).to(DEV)
        segs = mf.make_segments(b.n, b.k, b.x_off, b.y_off)
        y = torch.zeros(b.y_total, device=DEV)
        with torch.cuda.stream(stream):
            mf.mf_filter_batched(h, x, y, segs)              # sizes the workspace first
        stream.synchronize()
        ref = y.clone()
        y.zero_()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=stream):
            mf.mf_set_stream(h, torch.cuda.current_stream(DEV))
            mf.mf_filter_batched(h, x, y, segs)
        mf.mf_set_stream(h, stream)
        torch.cuda.synchronize(DEV)
        for _ in range(3):
            y.zero_()
            g.replay()
            torch.cuda.synchronize(DEV)
            assert torch.equal(y.view(torch.int32), ref.view(torch.int32))
        # an uncaptured call with other signals does not change what the graph does
        b2 = batched_signals(nseg=64, seed=9, n_hi=20_000)
        x2 = torch.from_numpy(b2.x).to(DEV)
        y2 = torch.zeros(b2.y_total, device=DEV)
        with torch.cuda.stream(stream):
            mf.mf_filter_batched(h, x2, y2, mf.make_segments(b2.n, b2.k, b2.x_off, b2.y_off))
        stream.synchronize()
        y.zero_()
        g.replay()
        torch.cuda.synchronize(DEV)
        assert torch.equal(y.view(torch.int32), ref.view(torch.int32))
    finally:
        mf.mf_destroy(h)
