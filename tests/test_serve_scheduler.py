"""Host logic of the continuous-batching request server (no GPU).

The scheduler runs against a simulated executor on a virtual clock: every
slot finishes a batch after a time proportional to its samples.  Checked:
every request completes once; the memory budget holds at every launch;
batches are homogeneous in dtype and tier and respect their size caps;
requests that arrive while other batches run are started before those
finish (continuous batching, not a queue drained batch by batch); FIFO order
within a class; idle workspaces are released when the oldest request does
not fit; a request above the whole budget is refused; percentiles.
"""
import numpy as np
import pytest

from paper_1406_1717_gb300.serve import AdmissionError, Scheduler, serve
from signals import Request, serving_requests


class VirtualClock:
    def __init__(self):
        self.t = 0.0

    def __call__(self):
        return self.t

    def wait(self, until):
        self.t = max(self.t, until)


class SimExecutor:
    def __init__(self, clock, ns_per_sample=1.0, overhead_s=20e-6):
        self.clock = clock
        self.ns = ns_per_sample
        self.overhead = overhead_s
        self.inflight = {}
        self.released = []
        self.launched = []

    def start(self):
        return 0.0

    def launch(self, b, now_s):
        dur = self.overhead + sum(j.n for j in b.jobs) * self.ns * 1e-9 * (4 if b.large else 1)
        b.handle = now_s + dur
        self.inflight[id(b)] = b
        self.launched.append((now_s, b))

    def done(self, b):
        return self.clock() >= b.handle

    def finish(self, b):
        return b.handle

    def retire(self, b):
        self.inflight.pop(id(b), None)

    def release(self, slot):
        self.released.append(slot)

    def next_event_s(self):
        return min((b.handle for b in self.inflight.values()), default=None)


def ws_model(slot, jobs):
    small = sum(8 * j.n for j in jobs if not j.large)
    big = max((40 * j.n for j in jobs if j.large), default=0)
    return max(small, big)


def large_of(k):
    return k >= 5001


def run(reqs, slots=4, budget=10 ** 9, **kw):
    clk = VirtualClock()
    ex = SimExecutor(clk)
    sch = Scheduler(slots, budget, ws_model, large_of, **kw)
    budgets = []
    orig = sch.form_batch

    def form(slot):
        b = orig(slot)
        budgets.append(sch.in_use())
        return b
    sch.form_batch = form
    rep = serve(reqs, ex, sch, clock=clk, wait=clk.wait)
    return rep, ex, sch, budgets


def test_trace_completes_within_budget():
    reqs = serving_requests(rate_hz=2000, duration_s=0.5, seed=3, n_hi=2e5)
    rep, ex, sch, budgets = run(reqs, slots=4, budget=2 * 10 ** 8)
    assert rep.requests == len(reqs)
    assert max(budgets) <= 2 * 10 ** 8
    assert sch.peak_bytes <= 2 * 10 ** 8
    assert np.all(rep.latencies_s > 0)
    seen = set()
    for _, b in ex.launched:
        assert len({j.dtype for j in b.jobs}) == 1
        assert len({j.large for j in b.jobs}) == 1
        assert len(b.jobs) <= (sch.max_large_jobs if b.large else sch.max_batch_jobs)
        for j in b.jobs:
            assert j.rid not in seen
            seen.add(j.rid)
    assert seen == {r.rid for r in reqs}
    s = rep.summary()
    assert s["p50_ms"] <= s["p99_ms"]
    assert s["requests"] == len(reqs)


def test_continuous_batching_overlaps_batches():
    # a long request first, then short ones arriving while it runs
    reqs = [Request(rid=0, arrival_s=0.0, n=4_000_000, k=101, dtype="float32", seed=1)]
    reqs += [Request(rid=i, arrival_s=1e-4 * i, n=10_000, k=31, dtype="float32", seed=i)
             for i in range(1, 20)]
    rep, ex, sch, _ = run(reqs, slots=2, budget=10 ** 9)
    first = ex.launched[0][1]
    assert [j.rid for j in first.jobs] == [0]
    later = [(t, b) for t, b in ex.launched[1:]]
    assert later and all(t < first.handle for t, _ in later[:3])
    short_done = max(j.done_s for _, b in later for j in b.jobs)
    assert short_done < first.handle          # short jobs finished while the long one ran


def test_fifo_within_a_class():
    reqs = serving_requests(rate_hz=5000, duration_s=0.2, seed=5, n_hi=1e5)
    rep, ex, sch, _ = run(reqs, slots=3, budget=10 ** 9)
    order = {}
    for t, b in ex.launched:
        for j in b.jobs:
            order.setdefault((j.dtype, j.large), []).append((t, j.arrival_s, j.rid))
    for cls, lst in order.items():
        starts = [a for _, a, _ in sorted(lst, key=lambda v: (v[0], v[1]))]
        assert starts == sorted(starts), cls


def test_budget_limits_concurrency_and_releases_idle_workspace():
    # L1 (large-k: io 8 MB, workspace 40 MB) on slot 0 and S1 (small) on slot 1;
    # S2 (io 24 MB, workspace 24 MB) arrives while L1 runs and does not fit
    # until L1 ends; then only after slot 0's idle 40 MB workspace is freed
    reqs = [Request(rid=0, arrival_s=0.0, n=1_000_000, k=9001, dtype="int32", seed=0),
            Request(rid=1, arrival_s=0.0, n=200_000, k=31, dtype="float32", seed=1),
            Request(rid=2, arrival_s=1e-3, n=3_000_000, k=31, dtype="float32", seed=2)]
    rep, ex, sch, budgets = run(reqs, slots=2, budget=60 * 10 ** 6)
    assert rep.requests == 3
    assert max(budgets) <= 60 * 10 ** 6
    assert ex.released == [0]
    start = {j.rid: t for t, b in ex.launched for j in b.jobs}
    l1 = next(b for _, b in ex.launched if b.jobs[0].rid == 0)
    assert start[2] >= l1.handle              # S2 waited for memory


def test_request_above_budget_is_refused():
    reqs = [Request(rid=0, arrival_s=0.0, n=10_000_000, k=20001, dtype="float32", seed=0)]
    with pytest.raises(AdmissionError):
        run(reqs, slots=2, budget=10 ** 8)


def test_batch_sample_cap():
    reqs = [Request(rid=i, arrival_s=0.0, n=300_000, k=31, dtype="float32", seed=i)
            for i in range(10)]
    rep, ex, sch, _ = run(reqs, slots=1, budget=10 ** 10, max_batch_samples=1_000_000)
    for _, b in ex.launched:
        assert sum(j.n for j in b.jobs) <= 1_000_000 or len(b.jobs) == 1
    assert rep.requests == 10
