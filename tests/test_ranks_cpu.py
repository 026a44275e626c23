"""The bench's multi-rank logic on CPU: two gloo ranks (the GPU runs use
NCCL with the same helpers).  Ranks are independent replicas: each draws its
own seed, the timed span is the slowest rank's, work adds up."""
import os
import socket
import sys

import pytest
import torch
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import bench
    dev = torch.device("cpu")
    dist = bench.init_ranks(world, dev)
    bench.barrier(dist)
    slowest = bench.max_over_ranks(dist, 1.5 + rank, dev)
    total = bench.sum_over_ranks(dist, 10.0 * (rank + 1), dev)
    seeds = [None] * world
    dist.all_gather_object(seeds, bench.replica_seed(7, rank))
    out[rank] = (slowest, total, tuple(seeds))
    dist.destroy_process_group()


def test_two_gloo_ranks():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        procs = [ctx.Process(target=_rank_main, args=(r, world, port, out))
                 for r in range(world)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
        assert all(p.exitcode == 0 for p in procs), [p.exitcode for p in procs]
        res = dict(out)
    for r in range(world):
        slowest, total, seeds = res[r]
        assert slowest == 2.5                  # the slowest replica's time
        assert total == 30.0                   # work of all replicas
        assert len(set(seeds)) == world        # every replica draws its own input


def test_one_rank_needs_no_group():
    sys.path.insert(0, ROOT)
    import bench
    dist = bench.init_ranks(1, torch.device("cpu"))
    assert dist is None
    assert bench.max_over_ranks(dist, 3.0, None) == 3.0
    assert bench.sum_over_ranks(dist, 3.0, None) == 3.0
    bench.barrier(dist)

