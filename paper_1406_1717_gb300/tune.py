"""Autotuner of the launch plans, per window-size class, and of the tier
crossover.

For each class of k (<= 64, <= 256, <= 1021, <= 2047, <= 4093) the tuner
chooses the block-sort variant (merge-sort tiles fused with the list
construction, or a warp radix sort with separate unwind and chain kernels;
Section 3 of the paper leaves the piecewise sort open, and both give the same
stable order), the number of block pairs per CTA of the sort kernel and of
the store kernel.  ``autotune`` times them on a seeded random-walk signal of
one representative k per class; ``tune_batched`` times them on the caller's
own batch, one class of its signals at a time.  Timing uses CUDA events (the
library's per-kernel events, mf_set_timing / mf_kernel_times, for the pairs
per CTA; the whole call for the variant).  The choices are applied with
mf_set_sort_variant and mf_set_tuning.  ``autotune`` also times both tiers
(shared-memory pipeline and large-k tier) at window sizes between 2047 and
the pipeline's limit and sets the handle's threshold (mf_set_tier_threshold)
to the smallest k from which the large-k tier is faster at every larger
candidate.  Results are cached as JSON (path from MF_TUNE_CACHE, default
paper_1406_1717_gb300/_tune_cache.json) and can be reloaded onto any handle
of the same GPU model.
"""
from __future__ import annotations

import json
import os

import torch

import numpy as np

from . import (make_segments, mf_filter, mf_filter_batched, mf_kernel_times, mf_set_sort_variant,
               mf_set_stream, mf_set_tier_threshold, mf_set_timing, mf_set_tuning, mf_sync)

CLASS_K = (63, 255, 1001, 2047, 4093)          # one representative k per class
CLASS_MAX = (64, 256, 1021, 2047, 4093, 1 << 30)   # largest k of each class
FUSED_MAX_K = 1021                             # merge-sort tiles serve k up to this
VARIANTS = (1, 2, 3)                           # merge-sort tiles, warp radix sort, adaptive tiles
TIER_K = (2047, 3001, 4095, 5001, 6001, 7001, 8001, 9343)
PIPELINE_ONLY = 1 << 30                        # threshold capped to the pipeline's limit
# 0 = the library's built-in choice (which may exceed every explicit value:
# the fused sort fills its warps' tiles, the store kernel covers about 8192
# outputs per CTA), so tuning never does worse than the built-in plan
SORT_CANDIDATES = (0, 1, 2, 3, 4, 6, 8, 12, 16, 24, 32, 48, 64, 128, 256)
STORE_CANDIDATES = (0, 1, 2, 4, 8, 16, 32, 64, 128)
_PKG = os.path.dirname(os.path.abspath(__file__))


def cache_path() -> str:
    return os.environ.get("MF_TUNE_CACHE", os.path.join(_PKG, "_tune_cache.json"))


def _time_groups(h, x, k, reps=5) -> dict:
    """Milliseconds per call of each kernel group (sort, unwind, chain, store)."""
    y = torch.empty(x.numel() - k + 1, dtype=x.dtype, device=x.device)
    mf_filter(h, x, k, y)                        # warm-up (and workspace)
    mf_set_timing(h, True)
    for _ in range(reps):
        mf_filter(h, x, k, y)
    mf_sync(h)
    t = mf_kernel_times(h, reps)
    mf_set_timing(h, False)
    return {g: v / reps for g, v in t.items()}


def _time_kernel(h, x, k, which, reps=5):
    return _time_groups(h, x, k, reps)[which]


def _time_call(h, x, k, reps=3):
    y = torch.empty(x.numel() - k + 1, dtype=x.dtype, device=x.device)
    mf_filter(h, x, k, y)
    mf_sync(h)
    start, stop = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    start.record()
    for _ in range(reps):
        mf_filter(h, x, k, y)
    stop.record()
    torch.cuda.synchronize(x.device)
    return start.elapsed_time(stop) / reps


def tune_tier_threshold(h, x, ks=TIER_K) -> dict:
    """Time both tiers at each k; returns {"threshold": k, "ms": {...}} and applies it."""
    times = {}
    for k in ks:
        mf_set_tier_threshold(h, PIPELINE_ONLY)
        tp = _time_call(h, x, k)
        mf_set_tier_threshold(h, 1)
        tl = _time_call(h, x, k)
        times[str(k)] = {"pipeline_ms": tp, "large_ms": tl}
    threshold = PIPELINE_ONLY
    for k in reversed(ks):
        if times[str(k)]["large_ms"] < times[str(k)]["pipeline_ms"]:
            threshold = k
        else:
            break
    mf_set_tier_threshold(h, threshold)
    return {"threshold": threshold, "ms": times}


def _tune_class(h, k, time_groups, time_total, variants) -> dict:
    """Choose (variant, sort pairs per CTA, store pairs per CTA) for the class
    of k: per variant the sort kernel's pairs per CTA by its own time, then the
    variant by the whole call, then the store kernel's pairs per CTA."""
    best = None
    for v in variants:                                   # the built-in choice is among them
        mf_set_sort_variant(h, k, v)
        best_g, best_t = 0, float("inf")
        for g in SORT_CANDIDATES:
            mf_set_tuning(h, k, g, 0)
            t = time_groups()
            t = t["sort"] + t["unwind"]                  # the radix variant unwinds apart
            if t < best_t:
                best_g, best_t = g, t
        mf_set_tuning(h, k, best_g, 0)
        total = time_total()
        if best is None or total < best[2]:
            best = (v, best_g, total)
    v, g, total = best
    mf_set_sort_variant(h, k, v)
    best_e, best_te = 0, float("inf")
    for e in STORE_CANDIDATES:
        mf_set_tuning(h, k, g, e)
        t = time_groups()["store"]
        if t < best_te:
            best_e, best_te = e, t
    mf_set_tuning(h, k, g, best_e)
    return {"sort_variant": v, "sort_pairs_per_cta": g, "store_pairs_per_cta": best_e,
            "call_ms": total, "store_ms": best_te}


def autotune(h, device=0, n=1 << 22, seed=20140607, classes=CLASS_K, tier=True) -> dict:
    """Tune every class on handle h; returns {k: {...}} and applies it."""
    from signals import random_walk_f32
    dev = torch.device("cuda", device)
    mf_set_stream(h, torch.cuda.current_stream(dev))
    x = torch.from_numpy(random_walk_f32(n, seed=seed)).to(dev)
    result = {}
    for k in classes:
        variants = VARIANTS if k <= FUSED_MAX_K else (0,)

        def groups(k=k):
            return _time_groups(h, x, k)

        result[str(k)] = _tune_class(h, k, groups, lambda k=k: _time_call(h, x, k), variants)
    if tier:
        result["tier"] = tune_tier_threshold(h, x)
    return result


def tune_batched(h, x, segs, reps=3) -> dict:
    """Tune the classes present in a batch on the batch itself: each class's
    signals are filtered alone (one batched call per candidate) and timed with
    CUDA events.  Applies the choices to h and returns {class k: {...}}."""
    segs = np.ascontiguousarray(segs)
    result = {}
    for kmax in CLASS_MAX:
        lo = 0 if kmax == CLASS_MAX[0] else CLASS_MAX[CLASS_MAX.index(kmax) - 1]
        sel = segs[(segs["k"] > lo) & (segs["k"] <= kmax)]
        if sel.size == 0:
            continue
        sub = sel.copy()
        m = sub["n"] - sub["k"] + 1
        sub["y_off"] = np.concatenate([[0], np.cumsum(m)[:-1]])
        y = torch.empty(int(m.sum()), dtype=x.dtype, device=x.device)

        def groups():
            mf_filter_batched(h, x, y, sub)
            mf_set_timing(h, True)
            for _ in range(reps):
                mf_filter_batched(h, x, y, sub)
            mf_sync(h)
            t = mf_kernel_times(h, reps)
            mf_set_timing(h, False)
            return {g: v / reps for g, v in t.items()}

        def total():
            mf_filter_batched(h, x, y, sub)
            mf_sync(h)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(reps):
                mf_filter_batched(h, x, y, sub)
            e1.record()
            torch.cuda.synchronize(x.device)
            return e0.elapsed_time(e1) / reps

        # the ordered-tile test (variant 3) serves 4-byte elements only
        variants = (VARIANTS if x.element_size() == 4 else (1, 2)) if kmax <= FUSED_MAX_K else (0,)
        result[str(kmax)] = {"signals": int(sel.size), **_tune_class(h, kmax, groups, total, variants)}
    return result


def save(result: dict, path: str = None) -> str:
    path = path or cache_path()
    meta = {"gpu": torch.cuda.get_device_name(0) if torch.cuda.is_available() else None,
            "classes": result}
    with open(path, "w") as f:
        json.dump(meta, f, indent=1)
    return path


def load(h, path: str = None) -> bool:
    """Apply a cached tuning to handle h; False if there is no cache."""
    path = path or cache_path()
    if not os.path.exists(path):
        return False
    with open(path) as f:
        meta = json.load(f)
    for k, v in meta.get("classes", {}).items():
        if k == "tier":
            mf_set_tier_threshold(h, int(v["threshold"]))
            continue
        mf_set_sort_variant(h, int(k), int(v.get("sort_variant", 0)))
        mf_set_tuning(h, int(k), int(v["sort_pairs_per_cta"]), int(v["store_pairs_per_cta"]))
    return True
