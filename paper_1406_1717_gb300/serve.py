"""Continuous-batching request server for median-filter jobs.

Requests (one signal each: n samples of int32 or float32, an odd window k)
arrive over time.  The server keeps a FIFO of arrived requests and a fixed
number of execution slots -- one CUDA stream and one library handle each.
Whenever a slot is free it forms a batch from the queue and launches it with
one ``mf_filter_batched`` call, so requests that arrive while others are on
the GPU join the next batch as soon as a slot and memory are free, and the
batches of different slots overlap on the device.

Admission is by a device-memory budget: the bytes in use are every slot's
workspace plus the input and output buffers of the batches in flight.  A
batch only takes a request if the budget still holds with that request's
buffers and the workspace growth it causes (``mf_batched_workspace_bytes``);
when the oldest request does not fit, the server frees idle slots'
workspaces, and otherwise waits for running batches to finish.

A batch holds requests of one dtype and of one tier (window sizes of the
shared-memory pipeline, or of the large-k tier), at most ``max_batch_jobs``
requests and ``max_batch_samples`` samples; large-k batches at most
``max_large_jobs`` requests, so that short jobs do not wait behind long ones.

Payloads are drawn on the device (``mf_fill_splitmix``, SplitMix64 seeded by
the request) in the request's input buffer, in the batch's stream, before
the filter.  Latency is completion minus arrival, with the completion time
taken from a CUDA event at the end of the batch.

The scheduling logic (``Scheduler``) is plain host code; ``serve`` runs it
against an executor -- ``CudaExecutor`` on a GPU, or any object with the same
methods (the tests use a simulated one on the CPU).
"""
from __future__ import annotations

import collections
import time
from dataclasses import dataclass, field

import numpy as np

DEFAULT_BUDGET = 40 * 10 ** 9


@dataclass
class Job:
    rid: int
    arrival_s: float
    n: int
    k: int
    dtype: str
    seed: int
    large: bool = False
    start_s: float = float("nan")
    done_s: float = float("nan")

    @property
    def m(self) -> int:
        return self.n - self.k + 1

    @property
    def io_bytes(self) -> int:
        return 4 * self.n + 4 * self.m


@dataclass
class Batch:
    slot: int
    dtype: str
    large: bool
    jobs: list = field(default_factory=list)
    io_bytes: int = 0
    ws_bytes: int = 0                 # slot workspace after this batch
    launch_s: float = float("nan")
    handle: object = None             # executor's record


class AdmissionError(RuntimeError):
    pass


class Scheduler:
    """FIFO queue, slots and the memory budget (no CUDA)."""

    def __init__(self, slots: int, budget_bytes: int, ws_need, large_of,
                 max_batch_jobs: int = 64, max_batch_samples: int = 1 << 26,
                 max_large_jobs: int = 2):
        self.slots = slots
        self.budget = int(budget_bytes)
        self.ws_need = ws_need            # (slot, [Job]) -> workspace bytes of one batched call
        self.large_of = large_of          # k -> runs on the large-k tier
        self.max_batch_jobs = max_batch_jobs
        self.max_batch_samples = max_batch_samples
        self.max_large_jobs = max_large_jobs
        self.queue = collections.deque()
        self.busy = [None] * slots        # Batch in flight per slot
        self.ws = [0] * slots             # workspace bytes each slot holds
        self.io_in_flight = 0
        self.peak_bytes = 0

    # -- accounting ------------------------------------------------------
    def in_use(self) -> int:
        return sum(self.ws) + self.io_in_flight

    def arrive(self, job: Job):
        job.large = bool(self.large_of(job.k))
        self.queue.append(job)

    def free_slots(self):
        return [s for s in range(self.slots) if self.busy[s] is None]

    def idle_workspace(self):
        """Slots without a batch in flight that still hold a workspace, largest first."""
        idle = [s for s in range(self.slots) if self.busy[s] is None and self.ws[s] > 0]
        return sorted(idle, key=lambda s: -self.ws[s])

    def _fits(self, slot: int, jobs, io: int) -> tuple:
        need = self.ws_need(slot, jobs)
        grow = max(0, need - self.ws[slot])
        return self.in_use() + io + grow <= self.budget, max(need, self.ws[slot])

    # -- batching --------------------------------------------------------
    def form_batch(self, slot: int):
        """Take requests for `slot` in FIFO order; None if nothing can start."""
        if self.busy[slot] is not None or not self.queue:
            return None
        head = self.queue[0]
        alone_need = self.ws_need(slot, [head])
        if head.io_bytes + alone_need > self.budget:
            raise AdmissionError(f"request {head.rid} (n={head.n}, k={head.k}) needs "
                                 f"{head.io_bytes + alone_need} bytes, above the budget")
        b = Batch(slot=slot, dtype=head.dtype, large=head.large)
        cap = self.max_large_jobs if head.large else self.max_batch_jobs
        samples = 0
        taken = []
        for idx, job in enumerate(self.queue):
            if len(b.jobs) >= cap:
                break
            if job.dtype != b.dtype or job.large != b.large:
                continue
            if b.jobs and samples + job.n > self.max_batch_samples:
                break
            ok, ws_after = self._fits(slot, b.jobs + [job], b.io_bytes + job.io_bytes)
            if not ok:
                break
            b.jobs.append(job)
            b.io_bytes += job.io_bytes
            b.ws_bytes = ws_after
            samples += job.n
            taken.append(idx)
        if not b.jobs:
            return None
        for idx in reversed(taken):
            del self.queue[idx]
        self.busy[slot] = b
        self.ws[slot] = b.ws_bytes
        self.io_in_flight += b.io_bytes
        self.peak_bytes = max(self.peak_bytes, self.in_use())
        return b

    def complete(self, b: Batch):
        self.busy[b.slot] = None
        self.io_in_flight -= b.io_bytes

    def release(self, slot: int):
        self.ws[slot] = 0

    def release_plan(self, slot: int):
        """Idle slots whose workspaces, freed largest first, let the oldest
        request start on `slot`; [] if freeing every idle workspace would not."""
        if not self.queue:
            return []
        head = self.queue[0]
        need = self.ws_need(slot, [head])
        ws = list(self.ws)
        plan = []
        for s in self.idle_workspace():
            ws[s] = 0
            plan.append(s)
            if sum(ws) + self.io_in_flight + head.io_bytes + max(0, need - ws[slot]) <= self.budget:
                return plan
        return []


@dataclass
class ServeReport:
    requests: int
    samples_out: int
    wall_s: float
    latencies_s: np.ndarray
    batches: int
    peak_bytes: int
    budget_bytes: int
    launch_s_per_batch: float

    @property
    def gsamples_per_s(self) -> float:
        return self.samples_out / self.wall_s / 1e9

    def percentile_ms(self, q: float) -> float:
        return float(np.percentile(self.latencies_s, q) * 1e3) if self.latencies_s.size else float("nan")

    def summary(self) -> dict:
        return {"requests": self.requests, "batches": self.batches,
                "output_samples": self.samples_out, "wall_s": round(self.wall_s, 3),
                "gsamples_per_s": round(self.gsamples_per_s, 4),
                "p50_ms": round(self.percentile_ms(50), 3),
                "p99_ms": round(self.percentile_ms(99), 3),
                "mean_ms": round(float(self.latencies_s.mean() * 1e3), 3) if self.latencies_s.size else None,
                "peak_device_bytes": int(self.peak_bytes), "budget_bytes": int(self.budget_bytes)}


def serve(requests, executor, scheduler: Scheduler, clock=time.perf_counter, wait=None,
          on_complete=None) -> ServeReport:
    """Run the request trace (sorted by arrival_s) to completion.

    executor: start() -> t0 (clock value of time 0); launch(batch, now_s);
    done(batch) -> bool; finish(batch) -> completion time in seconds since
    t0; release(slot); next_event_s() -> earliest time a running batch may
    finish (or None).  wait(until_s) blocks until that time (default: sleep
    on the clock).  on_complete(job, batch) is called for every finished job
    (the executor's buffers are still valid then).
    """
    reqs = sorted(requests, key=lambda r: r.arrival_s)
    t0 = executor.start()
    now = lambda: clock() - t0                                     # noqa: E731
    if wait is None:
        def wait(until_s):
            d = until_s - now()
            if d > 0:
                time.sleep(min(d, 2e-4))
    i = 0
    finished = []
    batches = 0
    launch_cost = 0.0
    while i < len(reqs) or scheduler.queue or any(b is not None for b in scheduler.busy):
        t = now()
        while i < len(reqs) and reqs[i].arrival_s <= t:
            r = reqs[i]
            scheduler.arrive(Job(rid=r.rid, arrival_s=r.arrival_s, n=r.n, k=r.k,
                                 dtype=r.dtype, seed=r.seed))
            i += 1
        progressed = False
        for b in [b for b in scheduler.busy if b is not None]:
            if executor.done(b):
                done_s = executor.finish(b)
                for job in b.jobs:
                    job.done_s = done_s
                    finished.append(job)
                    if on_complete is not None:
                        on_complete(job, b)
                executor.retire(b)
                scheduler.complete(b)
                progressed = True
        for slot in scheduler.free_slots():
            b = scheduler.form_batch(slot)
            if b is None and scheduler.queue:
                # the oldest request does not fit: free idle workspaces if that helps
                plan = scheduler.release_plan(slot)
                for s in plan:
                    executor.release(s)
                    scheduler.release(s)
                if plan:
                    b = scheduler.form_batch(slot)
            if b is None:
                break
            t_launch = now()
            for job in b.jobs:
                job.start_s = t_launch
            executor.launch(b, t_launch)
            launch_cost += now() - t_launch
            batches += 1
            progressed = True
        if not progressed:
            nxt = [reqs[i].arrival_s] if i < len(reqs) else []
            ev = executor.next_event_s()
            if ev is not None:
                nxt.append(ev)
            wait(min(nxt) if nxt else now())
    wall = max((j.done_s for j in finished), default=0.0)
    lat = np.array([j.done_s - j.arrival_s for j in finished], dtype=np.float64)
    return ServeReport(requests=len(finished), samples_out=sum(j.m for j in finished),
                       wall_s=wall, latencies_s=lat, batches=batches,
                       peak_bytes=scheduler.peak_bytes, budget_bytes=scheduler.budget,
                       launch_s_per_batch=launch_cost / max(batches, 1))


class CudaExecutor:
    """Slots = CUDA streams with one library handle each (GPU only)."""

    def __init__(self, slots: int, device: int = 0, tier_threshold: int = 0):
        import torch
        from . import mf_create, mf_set_tier_threshold
        self.torch = torch
        self.dev = torch.device("cuda", device)
        self.streams = [torch.cuda.Stream(self.dev) for _ in range(slots)]
        self.handles = [mf_create(device, s) for s in self.streams]
        for h in self.handles:
            if tier_threshold:
                mf_set_tier_threshold(h, tier_threshold)
        self.t0_event = None
        self.t0 = 0.0

    # sizes ---------------------------------------------------------------
    def segments(self, jobs):
        from . import make_segments
        n = np.array([j.n for j in jobs], dtype=np.int64)
        k = np.array([j.k for j in jobs], dtype=np.int64)
        x_off = np.concatenate([[0], np.cumsum(n)[:-1]]).astype(np.int64)
        m = n - k + 1
        y_off = np.concatenate([[0], np.cumsum(m)[:-1]]).astype(np.int64)
        return make_segments(n, k, x_off, y_off), int(n.sum()), int(m.sum()), x_off, y_off

    def ws_need(self, slot, jobs):
        from . import MF_FLOAT32, MF_INT32, mf_batched_workspace_bytes
        segs = self.segments(jobs)[0]
        code = MF_INT32 if jobs[0].dtype == "int32" else MF_FLOAT32
        return mf_batched_workspace_bytes(self.handles[slot], segs, code)

    def large_of(self, k):
        from . import tier_of
        return tier_of(self.handles[0], k) == "large"

    # serving -------------------------------------------------------------
    def start(self) -> float:
        torch = self.torch
        torch.cuda.synchronize(self.dev)
        self.t0_event = torch.cuda.Event(enable_timing=True)
        self.t0_event.record(torch.cuda.current_stream(self.dev))
        torch.cuda.synchronize(self.dev)
        self.t0 = time.perf_counter()
        return self.t0

    def launch(self, b: Batch, now_s: float):
        from . import mf_fill_splitmix, mf_filter_batched
        torch = self.torch
        segs, nx, ny, x_off, y_off = self.segments(b.jobs)
        dt = torch.int32 if b.dtype == "int32" else torch.float32
        stream = self.streams[b.slot]
        with torch.cuda.stream(stream):
            x = torch.empty(nx, dtype=dt, device=self.dev)
            y = torch.empty(ny, dtype=dt, device=self.dev)
            for j, off in zip(b.jobs, x_off):
                mf_fill_splitmix(x[int(off):int(off) + j.n], j.seed, stream)
            mf_filter_batched(self.handles[b.slot], x, y, segs)
            ev = torch.cuda.Event(enable_timing=True)
            ev.record(stream)
        b.handle = {"x": x, "y": y, "event": ev, "x_off": x_off, "y_off": y_off}

    def done(self, b: Batch) -> bool:
        return b.handle["event"].query()

    def finish(self, b: Batch) -> float:
        return self.t0_event.elapsed_time(b.handle["event"]) / 1e3

    def output(self, b: Batch, job: Job):
        idx = b.jobs.index(job)
        off = int(b.handle["y_off"][idx])
        return b.handle["y"][off:off + job.m]

    def retire(self, b: Batch):
        b.handle = None                   # buffers go back to torch's allocator

    def release(self, slot: int):
        from . import mf_release_workspace
        mf_release_workspace(self.handles[slot])

    def next_event_s(self):
        return None

    def close(self):
        from . import mf_destroy
        for h in self.handles:
            mf_destroy(h)
        self.handles = []


def run_trace(requests, slots: int = 8, budget_bytes: int = DEFAULT_BUDGET, device: int = 0,
              on_complete=None, **kw) -> ServeReport:
    """Serve a request trace on a GPU with a fresh executor."""
    ex = CudaExecutor(slots, device=device)
    try:
        sch = Scheduler(slots, budget_bytes, ex.ws_need, ex.large_of, **kw)
        return serve(requests, ex, sch, on_complete=(lambda j, b: on_complete(j, b, ex))
                     if on_complete else None)
    finally:
        ex.close()
