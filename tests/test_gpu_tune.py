"""Autotuner: tunes a class, applies and persists the choice; results stay
bit-exact under every tuned plan."""
import json

import numpy as np
import pytest
import torch

import oracle
import paper_1406_1717_gb300 as mf
from paper_1406_1717_gb300 import tune
from signals import random_walk_f32

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")


def test_autotune_one_class_and_reload(tmp_path):
    h = mf.mf_create(0, torch.cuda.current_stream(DEV))
    try:
        res = tune.autotune(h, n=1 << 18, classes=(255,), tier=False)
        assert set(res) == {"255"}
        g = res["255"]["sort_pairs_per_cta"]
        assert g in tune.SORT_CANDIDATES
        path = tune.save(res, str(tmp_path / "tune.json"))
        assert json.load(open(path))["classes"]["255"]["sort_pairs_per_cta"] == g
        h2 = mf.mf_create(0, torch.cuda.current_stream(DEV))
        try:
            assert tune.load(h2, path)
            x_np = random_walk_f32(50_003, seed=4)
            x = torch.from_numpy(x_np).to(DEV)
            for k in (201, 255):
                y = torch.empty(x_np.size - k + 1, device=DEV)
                mf.mf_filter(h2, x, k, y)
                mf.mf_sync(h2)
                ry, _ = oracle.median_filter(x_np, k)
                np.testing.assert_array_equal(y.cpu().numpy().view(np.uint32), ry.view(np.uint32))
        finally:
            mf.mf_destroy(h2)
    finally:
        mf.mf_destroy(h)


@pytest.mark.parametrize("g", [1, 2, 5, 13])
def test_every_sort_plan_is_exact(g):
    h = mf.mf_create(0, torch.cuda.current_stream(DEV))
    try:
        mf.mf_set_tuning(h, 1001, g, 3)
        x_np = random_walk_f32(60_011, seed=g)
        x = torch.from_numpy(x_np).to(DEV)
        y = torch.empty(x_np.size - 1001 + 1, device=DEV)
        mf.mf_filter(h, x, 1001, y)
        mf.mf_sync(h)
        ry, _ = oracle.median_filter(x_np, 1001)
        np.testing.assert_array_equal(y.cpu().numpy().view(np.uint32), ry.view(np.uint32))
    finally:
        mf.mf_destroy(h)


def test_tier_threshold_tuning_and_reload(tmp_path):
    h = mf.mf_create(0, torch.cuda.current_stream(DEV))
    try:
        x_np = random_walk_f32(1 << 20, seed=8)
        x = torch.from_numpy(x_np).to(DEV)
        res = tune.tune_tier_threshold(h, x, ks=(4095, 9343))
        assert res["threshold"] in (4095, 9343, tune.PIPELINE_ONLY)
        assert set(res["ms"]) == {"4095", "9343"}
        path = tune.save({"tier": res}, str(tmp_path / "tier.json"))
        h2 = mf.mf_create(0, torch.cuda.current_stream(DEV))
        try:
            assert tune.load(h2, path)
            xs = x_np[:40_000]
            xd = torch.from_numpy(xs).to(DEV)
            y = torch.empty(xs.size - 9343 + 1, device=DEV)
            mf.mf_filter(h2, xd, 9343, y)
            mf.mf_sync(h2)
            ry, _ = oracle.median_filter(xs, 9343)
            np.testing.assert_array_equal(y.cpu().numpy().view(np.uint32), ry.view(np.uint32))
        finally:
            mf.mf_destroy(h2)
    finally:
        mf.mf_destroy(h)


@pytest.mark.parametrize("variant", [1, 2, 3])
@pytest.mark.parametrize("k", [31, 255, 1001])
def test_both_sort_variants_are_exact(variant, k):
    """Merge-sort tiles (variant 1), the warp radix sort (variant 2) and the
    adaptive tiles (variant 3) give the same stable order, so the same outputs
    and argmedians as the oracle."""
    h = mf.mf_create(0, torch.cuda.current_stream(DEV))
    try:
        mf.mf_set_sort_variant(h, k, variant)
        x_np = random_walk_f32(40_009, seed=k + variant)
        x = torch.from_numpy(x_np).to(DEV)
        y = torch.empty(x_np.size - k + 1, device=DEV)
        a = torch.empty(x_np.size - k + 1, dtype=torch.int32, device=DEV)
        mf.mf_filter(h, x, k, y, a)
        mf.mf_sync(h)
        ry, ra = oracle.median_filter(x_np, k)
        np.testing.assert_array_equal(y.cpu().numpy().view(np.uint32), ry.view(np.uint32))
        np.testing.assert_array_equal(a.cpu().numpy().astype(np.int64), ra)
    finally:
        mf.mf_destroy(h)


def test_tune_batched_applies_choices_and_stays_exact():
    """Tuning on a batch picks a variant and pairs per CTA for every class the
    batch holds; the tuned batched call gives the untuned call's bits."""
    from signals import batched_signals
    b = batched_signals(nseg=200, seed=12, n_hi=40_000)
    x = torch.from_numpy(b.x).to(DEV)
    segs = mf.make_segments(b.n, b.k, b.x_off, b.y_off)
    h = mf.mf_create(0, torch.cuda.current_stream(DEV))
    try:
        y0 = torch.full((b.y_total,), -1.0, device=DEV)
        mf.mf_filter_batched(h, x, y0, segs)
        mf.mf_sync(h)
        res = tune.tune_batched(h, x, segs)
        present = {next(c for c in tune.CLASS_MAX if k <= c) for k in b.k}
        assert {int(c) for c in res} == present
        for c, v in res.items():
            assert v["sort_variant"] in ((1, 2, 3) if int(c) <= tune.FUSED_MAX_K else (0,))
            assert v["sort_pairs_per_cta"] in tune.SORT_CANDIDATES
        y1 = torch.full((b.y_total,), -2.0, device=DEV)
        mf.mf_filter_batched(h, x, y1, segs)
        mf.mf_sync(h)
        assert torch.equal(y0.view(torch.int32), y1.view(torch.int32))
    finally:
        mf.mf_destroy(h)
