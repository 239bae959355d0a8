"""Differentiation through the CUDA median filter (autograd wrapper).

* the gradient configuration: 64 float32 signals of n = 65,536, k = 63,
  distinct values (perm(0..n-1) * 1e-3 + N(0, 0.1)), upstream gradient N(0, 1):
  forward rows bit-exact against the oracle on sampled rows, backward against
  the oracle gradient (scatter of dL/dy to the argmedian) on every row;
* central finite differences in float64 on 8 signals of n = 256, k = 63,
  with a step below a quarter of the smallest gap between values, where the
  median filter is exactly linear in each input.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1406_1717_gb300.autograd import median_filter
from signals import distinct_f32

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")


def test_gradient_configuration_64x65536_k63():
    rows, n, k = 64, 65_536, 63
    x_np = np.stack([distinct_f32(n, seed=100 + r) for r in range(rows)])
    g_np = np.random.default_rng(1).standard_normal((rows, n - k + 1)).astype(np.float32)
    x = torch.from_numpy(x_np).to(DEV).requires_grad_(True)
    y, a = median_filter(x, k, return_argmed=True)
    y.backward(torch.from_numpy(g_np).to(DEV))
    gx = x.grad.cpu().numpy().astype(np.float64)
    y_np, a_np = y.detach().cpu().numpy(), a.cpu().numpy().astype(np.int64)
    for r in range(rows):
        if r % 8 == 0:
            ry, ra = oracle.median_filter(x_np[r], k)
            np.testing.assert_array_equal(y_np[r].view(np.uint32), ry.view(np.uint32))
            np.testing.assert_array_equal(a_np[r], ra)
        ref = oracle.median_gradient(g_np[r].astype(np.float64), a_np[r], n)
        bound = oracle.median_gradient(np.abs(g_np[r]).astype(np.float64), a_np[r], n)
        # each gx[j] is a float32 sum of at most k terms in a fixed order
        assert np.all(np.abs(gx[r] - ref) <= k * 6e-8 * bound + 1e-30)


def test_finite_differences_fp64():
    rows, n, k = 8, 256, 63
    rng = np.random.default_rng(7)
    for r in range(rows):
        x_np = distinct_f32(n, seed=500 + r)
        g = rng.standard_normal(n - k + 1)
        x = torch.from_numpy(x_np).to(DEV).requires_grad_(True)
        y = median_filter(x, k)
        y.backward(torch.from_numpy(g.astype(np.float32)).to(DEV))
        gx = x.grad.cpu().numpy().astype(np.float64)
        xd = x_np.astype(np.float64)
        gaps = np.diff(np.sort(xd))
        eps = 0.25 * gaps[gaps > 0].min()

        def loss(v):
            win = np.lib.stride_tricks.sliding_window_view(v, k)
            return float(np.dot(np.median(win, axis=1), g))

        fd = np.empty(n)
        for j in range(n):
            e = np.zeros(n)
            e[j] = eps
            fd[j] = (loss(xd + e) - loss(xd - e)) / (2 * eps)
        # the float32 upstream gradient rounds g; compare at float32 precision
        np.testing.assert_allclose(gx, fd, rtol=1e-5, atol=1e-5)
