"""The multi-GPU path is replicas only (a solve does not shard without collectives): each rank
solves its own instance and the bench reports the units of all ranks over the slowest rank's
time. The reduction is checked here with two gloo ranks on the CPU (no GPU), together with
the per-rank workloads the bench draws (different seeds give different instances)."""
import os
import sys

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _rank_main(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    import synth

    def red(op):
        def f(v):
            t = torch.tensor([v], dtype=torch.float64)
            dist.all_reduce(t, op=op)
            return float(t.item())
        return f

    # rank r: 10 ms per step for rank 0, 25 ms for rank 1; 3 steps of 300 iterations each
    ms = 10.0 if rank == 0 else 25.0
    value, ms_max = bench.replica_throughput(ms, 3 * 300, red(dist.ReduceOp.MAX), red(dist.ReduceOp.SUM))
    p = synth.large_noisy(seed=rank, m=64, n=256, s=4)
    g = [torch.zeros(4, dtype=torch.int64) for _ in range(world)]
    dist.all_gather(g, torch.from_numpy(p.support.astype(np.int64)))
    if rank == 0:
        torch.save({"value": value, "ms_max": ms_max, "supports": [t.numpy() for t in g]}, out)
    dist.barrier()
    dist.destroy_process_group()


def test_replica_throughput_over_two_gloo_ranks(tmp_path):
    out = str(tmp_path / "r.pt")
    port = 29500 + os.getpid() % 1000
    mp.start_processes(_rank_main, args=(2, port, out), nprocs=2, join=True, start_method="spawn")
    r = torch.load(out, weights_only=False)
    assert r["ms_max"] == 25.0
    assert r["value"] == pytest.approx(2 * 3 * 300 / 0.025)
    assert not np.array_equal(r["supports"][0], r["supports"][1])


def test_single_rank_is_the_identity():
    sys.path.insert(0, ROOT)
    import bench
    ident = lambda v: v
    value, ms_max = bench.replica_throughput(18.0, 300.0, ident, ident)
    assert ms_max == 18.0 and value == pytest.approx(300 / 0.018)
