"""Autotuner of the launch plans, per window-size class, and of the tier
crossover.

For each class of k (<= 64, <= 256, <= 1021, <= 2047, <= 4093) the tuner
times the candidate numbers of block pairs per CTA of the sort+merge kernel
and of the store kernel on a seeded random-walk signal, with the library's
CUDA-event kernel timing (mf_set_timing / mf_kernel_times), and applies the
fastest choice with mf_set_tuning.  It then times both tiers (shared-memory
pipeline and large-k tier) at window sizes between 2047 and the pipeline's
limit and sets the handle's threshold (mf_set_tier_threshold) to the
smallest k from which the large-k tier is faster at every larger candidate.
Results are cached as JSON (path from MF_TUNE_CACHE, default
paper_1406_1717_gb300/_tune_cache.json) and can be reloaded onto any handle
of the same GPU model.
"""
from __future__ import annotations

import json
import os

import torch

from . import (mf_filter, mf_kernel_times, mf_set_stream, mf_set_tier_threshold,
               mf_set_timing, mf_set_tuning, mf_sync)

CLASS_K = (63, 255, 1001, 2047, 4093)          # one representative k per class
TIER_K = (2047, 3001, 4095, 5001, 6001, 7001, 8001, 9343)
PIPELINE_ONLY = 1 << 30                        # threshold capped to the pipeline's limit
SORT_CANDIDATES = (1, 2, 3, 4, 6, 8, 12, 16, 24, 32, 48, 64)
STORE_CANDIDATES = (1, 2, 4, 8, 16)
_PKG = os.path.dirname(os.path.abspath(__file__))


def cache_path() -> str:
    return os.environ.get("MF_TUNE_CACHE", os.path.join(_PKG, "_tune_cache.json"))


def _time_kernel(h, x, k, which, reps=5):
    y = torch.empty(x.numel() - k + 1, dtype=x.dtype, device=x.device)
    mf_filter(h, x, k, y)                        # warm-up (and workspace)
    mf_set_timing(h, True)
    for _ in range(reps):
        mf_filter(h, x, k, y)
    mf_sync(h)
    t = mf_kernel_times(h, reps)[which] / reps
    mf_set_timing(h, False)
    return t


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


def autotune(h, device=0, n=1 << 22, seed=20140607, classes=CLASS_K, tier=True) -> dict:
    """Tune every class on handle h; returns {k: {...}} and applies it."""
    from signals import random_walk_f32
    dev = torch.device("cuda", device)
    mf_set_stream(h, torch.cuda.current_stream(dev))
    x = torch.from_numpy(random_walk_f32(n, seed=seed)).to(dev)
    result = {}
    for k in classes:
        best_g, best_t = 0, float("inf")
        for g in SORT_CANDIDATES:
            mf_set_tuning(h, k, g, 0)
            t = _time_kernel(h, x, k, "sort")
            if t < best_t:
                best_g, best_t = g, t
        best_e, best_te = 0, float("inf")
        for e in STORE_CANDIDATES:
            mf_set_tuning(h, k, best_g, e)
            t = _time_kernel(h, x, k, "store")
            if t < best_te:
                best_e, best_te = e, t
        mf_set_tuning(h, k, best_g, best_e)
        result[str(k)] = {"sort_pairs_per_cta": best_g, "store_pairs_per_cta": best_e,
                          "sort_ms": best_t, "store_ms": best_te}
    if tier:
        result["tier"] = tune_tier_threshold(h, x)
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
        mf_set_tuning(h, int(k), int(v["sort_pairs_per_cta"]), int(v["store_pairs_per_cta"]))
    return True
