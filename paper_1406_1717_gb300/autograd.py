"""torch.autograd wrapper of the median filter.

y = median_filter(x, k) picks, for every window, one input element (paper
Section 1: y_i is the median of x_i .. x_{i+k-1}); the library reports that
element's index (argmed).  Wherever the window's values are distinct, y_i is
locally the identity in x[argmed_i] and constant in the other inputs, so the
gradient of L with respect to x is gx[j] = sum of dL/dy_i over the outputs i
with argmed_i == j.  The forward pass keeps argmed; the backward pass runs the
library's deterministic gather kernel (mf_filter_backward).  Both passes run
in libmf.so; this module only marshals tensors.

x may be 1-D (one signal) or 2-D (rows filtered independently, same k).
"""
from __future__ import annotations

import numpy as np
import torch

from . import (default_handle, make_segments, mf_filter, mf_filter_backward,
               mf_filter_backward_rows, mf_filter_batched, mf_set_stream)


def _forward(x: torch.Tensor, k: int):
    dev = x.device.index
    h = default_handle(dev)
    mf_set_stream(h, torch.cuda.current_stream(x.device))
    if x.dim() == 1:
        m = x.numel() - k + 1
        y = torch.empty(m, dtype=x.dtype, device=x.device)
        a = torch.empty(m, dtype=torch.int32, device=x.device)
        mf_filter(h, x, k, y, a)
        return y, a
    rows, n = x.shape
    m = n - k + 1
    y = torch.empty((rows, m), dtype=x.dtype, device=x.device)
    a = torch.empty((rows, m), dtype=torch.int32, device=x.device)
    r = np.arange(rows, dtype=np.int64)
    segs = make_segments(np.full(rows, n), np.full(rows, k), r * n, r * m)
    mf_filter_batched(h, x, y, segs, a)
    return y, a


class MedianFilterFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, x: torch.Tensor, k: int):
        if not x.is_cuda or x.dtype != torch.float32:
            raise TypeError("median filter autograd needs a float32 CUDA tensor")
        x = x.contiguous()
        y, a = _forward(x, int(k))
        ctx.save_for_backward(a)
        ctx.k = int(k)
        ctx.shape = tuple(x.shape)
        ctx.mark_non_differentiable(a)
        return y, a

    @staticmethod
    def backward(ctx, gy: torch.Tensor, _ga=None):
        (a,) = ctx.saved_tensors
        k = ctx.k
        gy = gy.contiguous().to(torch.float32)
        h = default_handle(gy.device.index)
        mf_set_stream(h, torch.cuda.current_stream(gy.device))
        gx = torch.empty(ctx.shape, dtype=torch.float32, device=gy.device)
        if len(ctx.shape) == 1:
            mf_filter_backward(h, gy, a, ctx.shape[0], k, gx)
        else:
            mf_filter_backward_rows(h, gy, a.contiguous(), ctx.shape[0], ctx.shape[1], k, gx)
        return gx, None


def median_filter(x: torch.Tensor, k: int, return_argmed: bool = False):
    """Differentiable median filter (float32, CUDA); rows of a 2-D x independently."""
    y, a = MedianFilterFn.apply(x, k)
    return (y, a) if return_argmed else y
