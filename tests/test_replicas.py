"""The multi-GPU form is replicas only (independent volumes per rank, no data-path collective):
its host logic -- distinct per-rank volumes, the barrier, the slowest rank's time, the whole-job
value -- checked with two gloo processes on the CPU (127.0.0.1)."""
import os
import socket

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


def _rank_main(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms = 100.0 + 7.0 * rank  # rank 1 is the slowest
    dist.barrier()
    got = bench.max_over_ranks(ms, world, "cpu")
    seeds = [None] * world
    dist.all_gather_object(seeds, bench.rank_seed(rank))
    out[rank] = (got, bench.job_value(world, 1000, 30, got), seeds)
    dist.destroy_process_group()


def test_two_replicas_combine_the_slowest_time():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")  # never fork (a forked child of a CUDA process can hang)
    mgr = ctx.Manager()
    out = mgr.dict()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    for r in range(world):
        got, value, seeds = out[r]
        assert got == 107.0  # every rank sees the slowest rank's time
        assert value == pytest.approx(2 * 1000 * 30 / 0.107 / 1e9)
        assert len(set(seeds)) == world  # each replica decomposes its own volume


def test_single_process_needs_no_group():
    import bench
    assert bench.max_over_ranks(12.5, 1, "cpu") == 12.5
    assert bench.job_value(1, 134217728, 30, 409.3) == pytest.approx(134217728 * 30 / 0.4093 / 1e9)
