"""Run with MF_DEBUG=1 (the debug build of the library): every path of the
filter on small seeded inputs, each call compared with the oracle and followed
by mf_debug_take, which must report no failed device check.  Prints one JSON
object; used by tests/test_gpu_debug.py in a child process (the parent has
the normal build loaded)."""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402
import torch  # noqa: E402

import oracle  # noqa: E402
import paper_1406_1717_gb300 as mf  # noqa: E402
from signals import random_walk_f32, random_walk_f64, uniform_i32  # noqa: E402


def main():
    assert mf.DEBUG and mf.LIB_PATH.endswith("libmf_debug.so")
    dev = torch.device("cuda:0")
    h = mf.mf_create(0, torch.cuda.current_stream(dev))
    out = {"cases": [], "selftest": None}
    rng = np.random.default_rng(5)

    def check(name, x_np, k, rank=None, threshold=None):
        if threshold is not None:
            mf.mf_set_tier_threshold(h, threshold)
        x = torch.from_numpy(x_np).to(dev)
        m = x_np.size - k + 1
        y = torch.empty(m, dtype=x.dtype, device=dev)
        a = torch.empty(m, dtype=torch.int32, device=dev)
        if rank is None:
            mf.mf_filter(h, x, k, y, a)
            ry, ra = oracle.median_filter(x_np, k)
        else:
            mf.mf_filter_rank(h, x, k, rank, y, a)
            ry, ra = oracle.rank_filter(x_np, k, rank)
        mf.mf_sync(h)
        bits = np.uint64 if x_np.itemsize == 8 else np.uint32
        ok = (np.array_equal(y.cpu().numpy().view(bits), ry.view(bits))
              and np.array_equal(a.cpu().numpy().astype(np.int64), ra))
        cnt, site, val = mf.mf_debug_take(h)
        out["cases"].append({"name": name, "k": k, "n": int(x_np.size), "parity": bool(ok),
                             "failed_checks": cnt, "site": site, "value": val})
        if threshold is not None:
            mf.mf_set_tier_threshold(h, 0)

    ties = (uniform_i32(30011, seed=3) % 7).astype(np.int32)
    for k in (1, 3, 31, 63, 101, 255, 511, 1001, 1021):          # fused path
        check("float32 walk", random_walk_f32(max(20 * k, 5000) + 17, seed=k), k)
    check("int32 ties", ties, 31)
    check("int32 ties", ties, 1001)
    hi = (rng.integers(-2, 3, size=40_007).astype(np.int64) << 32) + rng.integers(0, 6, size=40_007)
    check("int64 high-half ties", hi, 101)
    check("float64 walk", random_walk_f64(50_021, seed=9), 1001)
    for k in (1023, 2047, 4093, 5001, 9343):                       # four-kernel pipeline
        check("float32 walk, pipeline", random_walk_f32(2 * k + 5 + 40_000 // k * k, seed=k), k,
              threshold=9345)
    check("float64 walk, pipeline", random_walk_f64(6 * 4095 + 3, seed=4), 4095, threshold=9345)
    for k in (5001, 10001):                                        # large-k tier
        check("float32 walk, large tier", random_walk_f32(2 * k + 77, seed=k), k)
    check("int32 ties, large tier", (uniform_i32(20_013, seed=8) % 5).astype(np.int32), 10001)
    check("rank filter, even k", ties, 64, rank=10)
    check("rank filter, large tier", random_walk_f32(24_033, seed=2), 12000, rank=11999)

    mf.mf_debug_selftest(h)
    out["selftest"] = list(mf.mf_debug_take(h))
    out["after_selftest"] = list(mf.mf_debug_take(h))
    mf.mf_destroy(h)
    print(json.dumps(out))


if __name__ == "__main__":
    main()
