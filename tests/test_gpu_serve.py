"""The request server on the GPU.

* payloads drawn on the device (SplitMix64) are bit-identical to the host
  generator in ``signals`` that feeds the oracle;
* a mixed trace (both dtypes, window sizes of both tiers, arrivals faster
  than one batch at a time) completes within the memory budget, and every
  request's result is bit-identical to the same request filtered alone;
* oracle spot checks on sampled windows of served requests.
"""
import numpy as np
import pytest
import torch

import oracle
import paper_1406_1717_gb300 as mf
from paper_1406_1717_gb300 import serve
from signals import Request, request_payload, serving_requests

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")


@pytest.mark.parametrize("dtype", ["int32", "float32"])
@pytest.mark.parametrize("seed", [0, 12345, 2 ** 63 + 7])
def test_device_payload_matches_host(dtype, seed):
    req = Request(rid=0, arrival_s=0.0, n=1_000_003, k=3, dtype=dtype, seed=seed)
    x = torch.empty(req.n, dtype=torch.int32 if dtype == "int32" else torch.float32, device=DEV)
    mf.mf_fill_splitmix(x, seed)
    torch.cuda.synchronize()
    host = request_payload(req)
    assert np.array_equal(x.cpu().numpy().view(np.uint32), host.view(np.uint32))


def test_mixed_trace_alone_equals_in_mix():
    reqs = serving_requests(rate_hz=3000, duration_s=0.05, seed=21, n_hi=3e5, k_hi=30001)
    reqs += [Request(rid=10_000, arrival_s=0.01, n=400_000, k=20001, dtype="int32", seed=77),
             Request(rid=10_001, arrival_s=0.01, n=250_000, k=9001, dtype="float32", seed=78)]
    assert len({r.dtype for r in reqs}) == 2
    outs = {}

    def keep(job, batch, ex):
        outs[job.rid] = ex.output(batch, job).cpu().numpy().copy()

    budget = 2 * 10 ** 9
    rep = serve.run_trace(reqs, slots=4, budget_bytes=budget, on_complete=keep)
    assert rep.requests == len(reqs) and rep.peak_bytes <= budget
    assert rep.batches < len(reqs)                       # requests were batched
    h = mf.mf_create(0, torch.cuda.current_stream(DEV))
    try:
        tiers = set()
        for r in reqs:
            dt = torch.int32 if r.dtype == "int32" else torch.float32
            x = torch.empty(r.n, dtype=dt, device=DEV)
            mf.mf_fill_splitmix(x, r.seed)
            y = torch.empty(r.n - r.k + 1, dtype=dt, device=DEV)
            mf.mf_filter(h, x, r.k, y)
            mf.mf_sync(h)
            assert np.array_equal(outs[r.rid].view(np.uint32), y.cpu().numpy().view(np.uint32)), r.rid
            tiers.add(mf.tier_of(h, r.k))
        assert tiers == {"pipeline", "large"}
    finally:
        mf.mf_destroy(h)
    rng = np.random.default_rng(0)
    for r in reqs[:: max(1, len(reqs) // 8)]:
        x = request_payload(r)
        m = r.n - r.k + 1
        st = np.unique(np.concatenate([[0, m - 1], rng.integers(0, m, 40)]))
        ry, _ = oracle.window_medians(x, r.k, st)
        assert np.array_equal(outs[r.rid][st].view(np.uint32), ry.view(np.uint32)), r.rid
