"""Multi-rank host logic on CPU with the gloo backend (world size 2):
the whole-job aggregation bench.py applies across replicas, and the
additivity of the count over a partition of endpoint vertices (the
sharding a multi-GPU count would use: each rank counts its starts, one sum
of two int64s)."""
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _init(rank, world, port):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    return dist


def _aggregation(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import bench
    dist = _init(rank, world, port)
    ms = [120.0, 150.0][rank]                     # rank 1 is the slowest
    slowest = bench.reduce_max(ms, dist, "cpu")
    out[rank] = (slowest, bench.whole_job_rate(1_000_000, world, slowest))
    dist.destroy_process_group()


def _shard(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import torch
    import oracle
    from paper_2308_07932_gb300 import synth
    dist = _init(rank, world, port)
    g = synth.chung_lu_scaled(41, 200_000)
    side = 1
    n = g.nV
    # contiguous start ranges, one per rank
    lo, hi = rank * n // world, (rank + 1) * n // world
    b, t, _, _ = oracle.sample_count(g, np.arange(lo, hi), side, threads=2)
    v = torch.tensor([b, t], dtype=torch.int64)
    dist.all_reduce(v)
    out[rank] = tuple(int(x) for x in v)
    dist.destroy_process_group()


def run_ranks(fn, world=2):
    import torch.multiprocessing as mp
    mgr = mp.Manager()
    out = mgr.dict()
    mp.start_processes(fn, args=(world, free_port(), out), nprocs=world, join=True,
                       start_method="spawn")
    return [out[r] for r in range(world)]


def test_whole_job_rate_takes_the_slowest_rank():
    res = run_ranks(_aggregation)
    for slowest, rate in res:
        assert slowest == 150.0
        assert rate == pytest.approx(2 * 1_000_000 / 0.150)


def test_start_partition_sums_to_the_full_count():
    import oracle
    from paper_2308_07932_gb300 import synth
    res = run_ranks(_shard)
    g = synth.chung_lu_scaled(41, 200_000)
    want = oracle.count(g, threads=4)
    for r in res:
        assert r == want
