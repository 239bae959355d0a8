"""Benchmark of the GB300 median filter: output Gsamples/s and % HBM roofline.

Workload (one step = one median filter of one signal, the whole hot path:
load, piecewise sort, pair post-processing, store):
  float32 Gaussian random walk, n = 2^26, k = 1001 (seeded, synthetic).
Also reported: the same n with int32 uniform [0, 2^31) (random input case).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun (N > 1) every rank filters its own signal (seed + rank): the
work is independent problems, weak scaling, no data-path collective; value
is the samples of all ranks over the slowest rank's time.

--impl reference times the CPU oracle (oracle/, per-window sort) on the host
cores, on a bounded sample of windows of the same workload per step.
"""
from __future__ import annotations

import argparse
import datetime as _dt
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N_SIG = 1 << 26
K_WIN = 1001
METRIC = "output Gsamples/s at n=2^26, k=1001 (float32 random walk)"
UNIT = "Gsamples/s"
WORKLOAD = "float32 Gaussian random walk, n=2^26, k=1001"
HBM_FALLBACK_GBS = 6800.0
KERNEL_SOURCES = ["paper_1406_1717_gb300/csrc/mf_device.cuh",
                  "paper_1406_1717_gb300/csrc/mf_tilesort.cuh",
                  "paper_1406_1717_gb300/csrc/mf_pipeline.cu",
                  "paper_1406_1717_gb300/csrc/mf_sortlist.cu"]
# CUDA kernel behind each timed group of the headline workload (4-byte
# elements, k = 1001: the fused path)
GROUP_KERNEL = {"sort": "sortlist_kernel", "unwind": "(none: made inside sortlist_kernel)",
                "chain": "chain_kernel<packed, words>", "store": "epilogue_kernel<u32>"}
# the same groups on the large-k tier (window-size overrides for profiling)
GROUP_KERNEL_LARGE = {"sort": "large_chunk_sort + large_merge tiers + large_ranks + large_jrank",
                      "unwind": "large_unwind", "chain": "large_seginit + large_chain",
                      "store": "large_epilogue"}
PROFILE_SUMMARY = os.path.join(ROOT, "profiles", "pipeline_randomwalk_n2p26_k1001.md")


# ---------------------------------------------------------------------------
# distributed helpers (host coordination only; no data-path collective)
# ---------------------------------------------------------------------------
def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def init_dist(ws, local, use_cuda):
    if ws <= 1:
        return None
    import torch
    import torch.distributed as dist
    backend = "nccl" if use_cuda else "gloo"
    if use_cuda:
        torch.cuda.set_device(local)
    dist.init_process_group(backend=backend)
    return dist


def barrier(dist, dev=None):
    if dist is not None:
        if dev is not None:
            dist.barrier(device_ids=[dev.index])
        else:
            dist.barrier()


def reduce_max(dist, value, dev=None):
    if dist is None:
        return value
    import torch
    t = torch.tensor([value], dtype=torch.float64, device=dev if dev is not None else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def weak_scaling_value(world_size, outputs_per_rank, steps, max_ms):
    """Whole-job throughput in Gsamples/s: every rank filters its own signal,
    so the job's outputs over the slowest rank's time."""
    return world_size * outputs_per_rank * steps / (max_ms * 1e-3) / 1e9


def rank_seed(base_seed, rank):
    """Each rank filters an independent signal drawn with base_seed + rank."""
    return base_seed + rank


# ---------------------------------------------------------------------------
def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return HBM_FALLBACK_GBS, "fallback"


def kernel_source_hash():
    h = hashlib.sha256()
    for rel in KERNEL_SOURCES:
        with open(os.path.join(ROOT, rel), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def profiled_traffic_total():
    """DRAM bytes per call of all the step's kernels (None unless every one is
    in the committed summary for the current source)."""
    parts = [profiled_traffic(g) for g in ("sort", "chain", "store")]
    return sum(parts) if all(v is not None for v in parts) else None


def profiled_traffic(kernel):
    """DRAM bytes per launch of `kernel` from the committed ncu summary, if it
    was taken on the current kernel source (else None)."""
    try:
        text = open(PROFILE_SUMMARY).read()
    except OSError:
        return None
    m_sha = re.search(r"kernel_source_sha:\s*([0-9a-f]+)", text)
    m_t = re.search(r"traffic_bytes_per_launch\[" + re.escape(kernel) + r"\]:\s*([0-9.eE+]+)", text)
    if not m_sha or not m_t or m_sha.group(1) != kernel_source_hash():
        return None
    return float(m_t.group(1))


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled during the timed region."""
    FIELDS = ("timestamp,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.dev = device_index
        self.proc = None
        self.file = None

    def start(self):
        try:
            self.file = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-i", str(self.dev), "-lms", "100"],
                stdout=self.file, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        time.sleep(0.3)

    def stop(self, t0, t1):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.15)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.file.flush()
        rows = []
        with open(self.file.name) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    ts = _dt.datetime.strptime(parts[0], "%Y/%m/%d %H:%M:%S.%f").timestamp()
                    rows.append((ts, float(parts[1]), float(parts[2]), parts[4:9]))
                except ValueError:
                    continue
        os.unlink(self.file.name)
        inside = [r for r in rows if t0 - 0.05 <= r[0] <= t1 + 0.05] or rows
        if not inside:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in inside for i, v in enumerate(r[3][1:5])
                          if v.lower() == "active"})
        return {"sm_mhz": statistics.median(r[1] for r in inside),
                "sm_max_mhz": max(r[2] for r in inside),
                "reasons": reasons, "samples": len(inside)}


def make_signal(kind, seed):
    from signals import random_walk_f32, random_walk_f64, uniform_i32
    if kind == "walk":
        return random_walk_f32(N_SIG, seed=seed)
    if kind == "walk64":
        return random_walk_f64(N_SIG, seed=seed)
    return uniform_i32(N_SIG, seed=seed)


def cpu_oracle_rate(x, k, target_s, seed=0):
    """Oracle windows/s on a bounded random sample of windows (all host cores)."""
    import oracle
    rng = np.random.default_rng(seed)
    m = x.size - k + 1
    pilot = rng.integers(0, m, size=4000)
    t = time.perf_counter()
    oracle.window_medians(x, k, pilot)
    dt = max(time.perf_counter() - t, 1e-6)
    count = int(max(4000, min(50_000_000, 4000 * target_s / dt)))
    starts = rng.integers(0, m, size=count)
    t = time.perf_counter()
    oracle.window_medians(x, k, starts)
    dt = time.perf_counter() - t
    return count / dt, count, dt, oracle.max_threads()


# ---------------------------------------------------------------------------
def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    from signals import DEFAULT_SEED
    x = make_signal("walk", DEFAULT_SEED)
    import oracle
    oracle.build()
    rng = np.random.default_rng(1)
    m = x.size - K_WIN + 1
    per_step = args.ref_windows
    for _ in range(args.warmup):
        oracle.window_medians(x, K_WIN, rng.integers(0, m, size=per_step))
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.window_medians(x, K_WIN, rng.integers(0, m, size=per_step))
    dt = time.perf_counter() - t0
    value = per_step * args.steps / dt / 1e9
    cores = oracle.max_threads()
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": dt / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "n": N_SIG, "k": K_WIN,
                   "sample": f"{per_step} random windows per step"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"{per_step} random windows of the workload per step, "
                                   f"{args.steps} steps"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def run_ours(args):
    import torch
    ws, rank, local = dist_env()
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA GPU")
    dist = init_dist(ws, local, True)
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    import paper_1406_1717_gb300 as mf
    if not os.path.exists(mf.LIB_PATH):
        import __graft_entry__
        __graft_entry__.build()
    from signals import DEFAULT_SEED
    seed = rank_seed(DEFAULT_SEED, rank)

    stream = torch.cuda.Stream(dev)
    h = mf.mf_create(dev.index, stream)
    k = K_WIN
    m = N_SIG - k + 1

    def device_run(kind):
        x_np = make_signal(kind, seed)
        x = torch.from_numpy(x_np).to(dev)
        y = torch.empty(m, dtype=x.dtype, device=dev)
        with torch.cuda.stream(stream):
            for _ in range(args.warmup):
                mf.mf_filter(h, x, k, y)
        stream.synchronize()
        barrier(dist, dev)
        torch.cuda.synchronize(dev)
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
        mf.mf_set_timing(h, True)
        launches0 = mf.mf_launch_count(h)
        t_wall0 = time.time()
        with torch.cuda.stream(stream):
            ev[0].record(stream)
            for s in range(args.steps):
                mf.mf_filter(h, x, k, y)
                ev[s + 1].record(stream)
        stream.synchronize()
        torch.cuda.synchronize(dev)
        t_wall1 = time.time()
        barrier(dist, dev)
        launches = mf.mf_launch_count(h) - launches0
        per = [ev[s].elapsed_time(ev[s + 1]) for s in range(args.steps)]
        total_ms = ev[0].elapsed_time(ev[-1])
        ncalls = min(args.steps, 128)
        kt = {name: v / ncalls for name, v in mf.mf_kernel_times(h, ncalls).items()}
        mf.mf_set_timing(h, False)
        del x, y
        return x_np, total_ms, per, launches, (t_wall0, t_wall1), kt

    sampler = ClockSampler(dev.index)
    sampler.start()
    x_walk, total_ms, per, launches, win, kt = device_run("walk")
    clocks = sampler.stop(*win)
    total_ms_max = reduce_max(dist, total_ms, dev)
    ms_per_step = total_ms_max / args.steps
    value = weak_scaling_value(ws, m, args.steps, total_ms_max)

    # int32 uniform variant of the same size (random-input case)
    _, total_i, per_i, _, _, kt_i = device_run("int")
    total_i = reduce_max(dist, total_i, dev)
    value_int = weak_scaling_value(ws, m, args.steps, total_i)
    # float64 random walk of the same length (64-bit keys)
    _, total_d, per_d, _, _, kt_d = device_run("walk64")
    total_d = reduce_max(dist, total_d, dev)
    value_f64 = weak_scaling_value(ws, m, args.steps, total_d)

    # end to end through the host-buffer entry point (pinned host memory)
    xh = torch.from_numpy(x_walk).pin_memory()
    yh = torch.empty(m, dtype=torch.float32).pin_memory()
    xh_np, yh_np = xh.numpy(), yh.numpy()
    e2e_steps = max(3, min(args.steps, 20))
    mf.mf_filter_host(h, xh_np, k, yh_np)
    barrier(dist, dev)
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        mf.mf_filter_host(h, xh_np, k, yh_np)
    e2e_s = reduce_max(dist, time.perf_counter() - t0, dev)
    e2e_value = ws * m * e2e_steps / e2e_s / 1e9

    batched = None if args.skip_extra else bench_batched(mf, h, dev, stream, seed, args)
    gradient = None if args.skip_extra else bench_gradient(dev, stream, seed, args)
    serving = None
    if not args.skip_extra and ws == 1 and args.serve_seconds > 0:
        serving = bench_serving(dev, DEFAULT_SEED, args)

    small = None
    if not args.skip_extra:
        try:
            small = bench_small(mf, h, dev, stream, args)
        except Exception as exc:                   # reported, the headline line still prints
            small = {"error": f"{type(exc).__name__}: {exc}"}

    peak, peak_kind = peaks()
    alg_bytes = 4 * N_SIG + 4 * m
    # the whole step (every kernel of the call) against the algorithmic bytes
    achieved = alg_bytes / (ms_per_step * 1e-3) / 1e9
    dom = max(kt, key=kt.get)                     # dominant kernel, CUDA-event average
    kernel_ms = kt[dom]
    # the committed DRAM bytes were taken on the n = 2^26, k = 1001 workload
    headline = N_SIG == 1 << 26 and K_WIN == 1001
    dom_traffic = profiled_traffic(dom) if headline else None

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        rate, count, dt, cores = cpu_oracle_rate(x_walk, k, args.cpu_seconds)
        cpu = {"value": rate / 1e9, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": f"{count} random windows of the workload ({dt:.1f} s of CPU work)"}

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "n": N_SIG, "k": k, "signal_dtype": "float32",
                   "seed": DEFAULT_SEED, "per_rank": "independent signal (seed + rank)",
                   "l2": (f"inputs larger than L2 ({4 * N_SIG / 1e6:.0f} MB input vs 129 MB L2), "
                          "no flush") if 4 * N_SIG > 129e6 else
                         f"input {4 * N_SIG / 1e6:.0f} MB fits in L2: profiling size only",
                   "parallelism": f"replicas x{ws}"},
        "p50_ms": float(np.percentile(per, 50)), "p99_ms": float(np.percentile(per, 99)),
        "int32_uniform": {"value": value_int, "unit": UNIT,
                          "ms_per_step": total_i / args.steps,
                          "p50_ms": float(np.percentile(per_i, 50)), "kernels_ms": kt_i},
        "float64_random_walk": {"value": value_f64, "unit": UNIT,
                                "ms_per_step": total_d / args.steps,
                                "p50_ms": float(np.percentile(per_d, 50)), "kernels_ms": kt_d},
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": 4 * N_SIG,
                "d2h_bytes_per_step": 4 * m, "steps": e2e_steps,
                "entry": "mf_filter_host (pinned host buffers)"},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": profiled_traffic_total() if headline else None,
                     "scope": "whole step: algorithmic bytes (x read once, y written once) "
                              "over ms_per_step; traffic = DRAM bytes of all the step's kernels",
                     "peak_source": f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs)",
                     "algorithmic_bytes_per_launch": alg_bytes,
                     "dominant_kernel": {
                         "kernel": (GROUP_KERNEL_LARGE if mf.tier_of(h, k) == "large"
                                    else GROUP_KERNEL).get(dom, dom), "kernel_ms": kernel_ms,
                         "share": kernel_ms / ms_per_step,
                         "traffic": dom_traffic,
                         "traffic_gbs": (dom_traffic / (kernel_ms * 1e-3) / 1e9
                                         if dom_traffic else None),
                         "dominant_kernel_frac": (dom_traffic / (kernel_ms * 1e-3) / 1e9 / peak
                                                  if dom_traffic else None),
                         "note": "dominant_kernel_frac = the kernel's own DRAM bytes (ncu) "
                                 "over its CUDA-event time, against the same peak"}},
        "kernels_ms": kt,
        "small_uniform_k31": small,
        "batched": batched,
        "gradient": gradient,
        "serving": serving,
        "clocks": clocks,
        "gpu_launches": launches,
        "cpu_baseline": cpu,
    }
    mf.mf_destroy(h)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


def bench_small(mf, h, dev, stream, args):
    """n = 100,000 float32 U[0,1), k = 31: a launch-latency-bound size.

    Device time: 1000 calls of mf_filter captured in one CUDA graph, each on
    its own copy of the signal and its own output (400 MB in and 400 MB out
    over the graph, more than L2, so no call finds its input in L2); the graph
    is replayed and timed with CUDA events, kernel time = graph time / 1000.
    p50 / p99: the same calls launched one by one behind a sleep kernel (so
    the queue is full and no launch gap is timed), CUDA events between calls.
    End to end: mf_filter_host with pinned host buffers (copies in, filter,
    copies out, synchronised), wall time per call."""
    import torch
    from signals import uniform_f32
    n, k, calls = 100_000, 31, 1000
    m = n - k + 1
    x_np = uniform_f32(n)
    xs = torch.from_numpy(x_np).to(dev).repeat(calls).view(calls, n)
    ys = torch.empty((calls, m), dtype=torch.float32, device=dev)
    with torch.cuda.stream(stream):
        for c in range(3):
            mf.mf_filter(h, xs[c], k, ys[c])
    stream.synchronize()
    l0 = mf.mf_launch_count(h)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=stream):
        mf.mf_set_stream(h, torch.cuda.current_stream(dev))
        for c in range(calls):
            mf.mf_filter(h, xs[c], k, ys[c])
    launches_per_call = (mf.mf_launch_count(h) - l0) / calls
    mf.mf_set_stream(h, stream)
    reps = 3
    with torch.cuda.stream(stream):
        g.replay()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            g.replay()
        e1.record(stream)
    stream.synchronize()
    graph_call_ms = e0.elapsed_time(e1) / (reps * calls)
    del g
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(calls + 1)]
    with torch.cuda.stream(stream):
        torch.cuda._sleep(200_000_000)
        ev[0].record(stream)
        for c in range(calls):
            mf.mf_filter(h, xs[c], k, ys[c])
            ev[c + 1].record(stream)
    stream.synchronize()
    per = [ev[c].elapsed_time(ev[c + 1]) for c in range(calls)]
    xh = torch.from_numpy(x_np).pin_memory()
    yh = torch.empty(m, dtype=torch.float32).pin_memory()
    xh_np, yh_np = xh.numpy(), yh.numpy()
    for _ in range(5):
        mf.mf_filter_host(h, xh_np, k, yh_np)
    wall = []
    for _ in range(calls):
        t0 = time.perf_counter()
        mf.mf_filter_host(h, xh_np, k, yh_np)
        wall.append((time.perf_counter() - t0) * 1e3)
    e2e_ms = float(np.mean(wall))
    del xs, ys
    return {"workload": "float32 U[0,1), n=100000, k=31 (99970 outputs)",
            "value": m / (graph_call_ms * 1e-3) / 1e9, "unit": UNIT,
            "kernel_ms": graph_call_ms, "launches_per_call": launches_per_call,
            "timing": "CUDA graph of 1000 calls on 1000 copies of the signal (inputs and "
                      "outputs 400 MB each, larger than L2), replayed 3 times",
            "p50_ms": float(np.percentile(per, 50)), "p99_ms": float(np.percentile(per, 99)),
            "p_timing": "1000 calls queued behind a sleep kernel, CUDA events between calls",
            "e2e": {"value": m / (e2e_ms * 1e-3) / 1e9, "unit": UNIT, "mean_ms": e2e_ms,
                    "p50_ms": float(np.percentile(wall, 50)),
                    "p99_ms": float(np.percentile(wall, 99)),
                    "h2d_bytes_per_step": 4 * n, "d2h_bytes_per_step": 4 * m,
                    "entry": "mf_filter_host (pinned host buffers), wall time per call"}}


def bench_batched(mf, h, dev, stream, seed, args):
    """4096 signals of log-uniform n and k in one batched call (captured in a
    CUDA graph and replayed) against a loop of per-signal calls.  The graph is
    timed with the built-in launch plans and again after the autotuner has
    chosen each class's sort variant and pairs per CTA on this batch."""
    import torch
    from paper_1406_1717_gb300 import tune
    from signals import batched_signals
    b = batched_signals(nseg=4096, seed=seed)
    x = torch.from_numpy(b.x).to(dev)
    y = torch.empty(b.y_total, dtype=torch.float32, device=dev)
    segs = mf.make_segments(b.n, b.k, b.x_off, b.y_off)
    reps = max(3, min(args.steps, 10))

    def graph_time():
        with torch.cuda.stream(stream):
            mf.mf_filter_batched(h, x, y, segs)
        stream.synchronize()
        l0 = mf.mf_launch_count(h)
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=stream):
            mf.mf_set_stream(h, torch.cuda.current_stream(dev))
            mf.mf_filter_batched(h, x, y, segs)
        launches = mf.mf_launch_count(h) - l0
        mf.mf_set_stream(h, stream)
        with torch.cuda.stream(stream):
            for _ in range(2):
                g.replay()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(reps):
                g.replay()
            e1.record(stream)
        stream.synchronize()
        return e0.elapsed_time(e1) / reps, launches

    builtin_ms, _ = graph_time()
    with torch.cuda.stream(stream):
        tuned = tune.tune_batched(h, x, segs)
    stream.synchronize()
    graph_ms, launches_per_call = graph_time()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(stream):
        e0.record(stream)
        for _ in range(reps):
            mf.mf_filter_batched(h, x, y, segs)
        e1.record(stream)
    stream.synchronize()
    batched_ms = e0.elapsed_time(e1) / reps
    ys = [torch.empty(int(b.n[s] - b.k[s] + 1), device=dev) for s in range(len(b.n))]
    xs = [x[int(b.x_off[s]):int(b.x_off[s] + b.n[s])] for s in range(len(b.n))]
    with torch.cuda.stream(stream):
        e0.record(stream)
        for s in range(len(b.n)):
            mf.mf_filter(h, xs[s], int(b.k[s]), ys[s])
        e1.record(stream)
    stream.synchronize()
    loop_ms = e0.elapsed_time(e1)
    return {"workload": "4096 float32 signals, n log-uniform [1e3, 262144], odd k log-uniform "
                        "[3, 4095], 10% +-1e3 impulses",
            "outputs": int(b.y_total), "graph_ms": graph_ms, "batched_ms": batched_ms,
            "graph_ms_builtin_plans": builtin_ms,
            "tuned": {c: {kk: v[kk] for kk in ("signals", "sort_variant", "sort_pairs_per_cta",
                                                "store_pairs_per_cta")}
                      for c, v in tuned.items()},
            "per_signal_loop_ms": loop_ms, "launches_per_batched_call": int(launches_per_call),
            "value_graph": b.y_total / (graph_ms * 1e-3) / 1e9,
            "value_per_signal": b.y_total / (loop_ms * 1e-3) / 1e9, "unit": UNIT,
            "speedup_vs_per_signal": loop_ms / graph_ms}


def bench_serving(dev, seed, args):
    """Poisson arrivals at 2000 requests/s (n log-uniform [1e3, 1e7], odd k
    log-uniform [3, 100001], int32 or float32 payloads drawn on the device),
    served with continuous batching on 8 streams under a 40 GB device-memory
    budget; the first seconds of the same trace also through a per-request
    server (one stream, one request per call) for comparison."""
    from paper_1406_1717_gb300 import serve
    from signals import serving_requests
    reqs = serving_requests(duration_s=args.serve_seconds, seed=seed)
    offered = sum(r.n - r.k + 1 for r in reqs) / args.serve_seconds / 1e9
    rep = serve.run_trace(reqs, slots=8, budget_bytes=serve.DEFAULT_BUDGET, device=dev.index)
    out = {"workload": f"Poisson 2000 req/s for {args.serve_seconds:g} s, n log-uniform "
                       "[1e3, 1e7], odd k log-uniform [3, 100001], int32 U[0,65536) or float32 "
                       "U[0,1) (SplitMix64 on the device), budget 40 GB, 8 streams",
           "offered_gsamples_per_s": offered, "unit": UNIT, "continuous": rep.summary()}
    cut = min(args.serve_seconds, args.serve_baseline_seconds)
    if cut > 0:
        head = [r for r in reqs if r.arrival_s < cut]
        per = serve.run_trace(head, slots=1, budget_bytes=serve.DEFAULT_BUDGET,
                              device=dev.index, max_batch_jobs=1, max_large_jobs=1)
        out["per_request_first_seconds"] = {"seconds": cut, **per.summary()}
    return out


def bench_gradient(dev, stream, seed, args):
    """Forward (with argmedian) and backward of 64 float32 signals, n = 65536,
    k = 63, distinct values, upstream gradient N(0, 1)."""
    import torch
    from paper_1406_1717_gb300.autograd import median_filter
    from signals import distinct_f32
    rows, n, k = 64, 65536, 63
    x = torch.from_numpy(np.stack([distinct_f32(n, seed=seed + r) for r in range(rows)])).to(dev)
    gy = torch.from_numpy(np.random.default_rng(seed).standard_normal((rows, n - k + 1))
                          .astype(np.float32)).to(dev)
    reps = max(3, min(args.steps, 10))
    with torch.cuda.stream(stream):
        for it in range(reps + 2):
            if it == 2:
                e0 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
            xr = x.detach().requires_grad_(True)
            y = median_filter(xr, k)
            y.backward(gy)
        e1 = torch.cuda.Event(enable_timing=True)
        e1.record(stream)
    stream.synchronize()
    ms = e0.elapsed_time(e1) / reps
    return {"workload": "64 x 65536 float32, k=63, forward + backward", "fwd_bwd_ms": ms,
            "value": rows * (n - k + 1) / (ms * 1e-3) / 1e9, "unit": UNIT}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--ref-windows", type=int, default=100_000)
    ap.add_argument("--skip-extra", action="store_true",
                    help="skip the batched, gradient and serving configurations")
    ap.add_argument("--serve-seconds", type=float, default=60.0,
                    help="length of the served request trace (0 = skip)")
    ap.add_argument("--serve-baseline-seconds", type=float, default=10.0,
                    help="first seconds of the trace also served one request at a time")
    ap.add_argument("--n", type=int, default=0,
                    help="signal length override for profiling captures (default 2^26)")
    ap.add_argument("--k", type=int, default=0,
                    help="window override for profiling captures (default 1001)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.n or args.k:
        global N_SIG, K_WIN, WORKLOAD
        N_SIG = args.n or N_SIG
        K_WIN = args.k or K_WIN
        WORKLOAD = (f"float32 Gaussian random walk, n={N_SIG}, k={K_WIN} "
                    "(size override, not the headline workload)")
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
