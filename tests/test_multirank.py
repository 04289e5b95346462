"""The multi-rank bench path on CPU with gloo (world size 2): each rank solves its own instance,
the job time is the slowest rank's, and throughput counts every rank's unknowns."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms = 100.0 * (rank + 1)                      # rank 1 is the slow one
        worst = bench.max_over_ranks(ms)
        seeds = [None] * world
        dist.all_gather_object(seeds, bench.rank_seed(rank))
        out[rank] = (worst, bench.job_throughput(1000, world, worst), tuple(seeds))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks():
    world = 2
    port = _free_port()
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_worker, args=(world, port, out), nprocs=world, start_method="spawn", join=True)
    for r in range(world):
        worst, thr, seeds = out[r]
        assert worst == 200.0                         # max over ranks, identical everywhere
        assert thr == pytest.approx(1000 * 2 / 0.2)   # both ranks' unknowns over the slowest time
        assert len(set(seeds)) == world               # distinct instances per rank


def test_single_process_is_identity():
    assert bench.max_over_ranks(42.0) == 42.0
    assert bench.job_throughput(10, 1, 1000.0) == 10.0
