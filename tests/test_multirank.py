"""The bench's N > 1 path on CPU: two gloo ranks, the host-side coordination
bench.py uses under torchrun (barrier, max over ranks of the timed region,
whole-job weak-scaling throughput, one independent signal per rank).  No
data-path collective exists: ranks only exchange their timings."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, results):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import bench
    ws, r, local = bench.dist_env()
    assert (ws, r, local) == (world, rank, rank)
    d = bench.init_dist(ws, local, use_cuda=False)
    try:
        bench.barrier(d)
        local_ms = 10.0 + 5.0 * rank                     # rank 1 is the slower rank
        mx = bench.reduce_max(d, local_ms)
        value = bench.weak_scaling_value(ws, 1000, 4, mx)
        from signals import random_walk_f32
        sig = random_walk_f32(64, seed=bench.rank_seed(7, rank))
        digest = torch.tensor([float(sig.astype(np.float64).sum())], dtype=torch.float64)
        gathered = [torch.zeros(1, dtype=torch.float64) for _ in range(ws)]
        dist.all_gather(gathered, digest)
        results[rank] = (mx, value, [float(g.item()) for g in gathered])
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_weak_scaling():
    world = 2
    port = _free_port()
    manager = mp.Manager()
    results = manager.dict()
    mp.spawn(_worker, args=(world, port, results), nprocs=world, join=True)
    assert set(results.keys()) == {0, 1}
    for rank in range(world):
        mx, value, digests = results[rank]
        assert mx == pytest.approx(15.0)                 # max over ranks, not the local time
        assert value == pytest.approx(2 * 1000 * 4 / 15e-3 / 1e9)
        assert digests[0] != digests[1]                  # independent signals per rank


def test_single_rank_needs_no_process_group():
    import bench
    assert bench.init_dist(1, 0, use_cuda=False) is None
    assert bench.reduce_max(None, 3.5) == 3.5
    assert bench.weak_scaling_value(1, 10, 2, 1.0) == pytest.approx(2e-5)
