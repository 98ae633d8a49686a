"""The multi-GPU form of the bench is replicas only: each rank advances its own
system with its own seed, and the whole-job rate is the steps of all ranks over
the slowest rank's time.  The reduction and the aggregation are host logic,
tested here with two gloo ranks on the CPU (no GPU, no NCCL)."""
from __future__ import annotations

import os
import socket

import pytest
import torch.multiprocessing as mp

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    os.environ["RANK"] = str(rank)
    os.environ["WORLD_SIZE"] = str(world)
    os.environ["LOCAL_RANK"] = str(rank)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    r, w, loc = bench.dist_env()
    local_s = 2.0 + r                       # rank 1 is the slower one
    slowest = bench.max_over_ranks(local_s, w, device="cpu")
    q.put((r, w, loc, slowest, bench.whole_job_rate(1000, slowest, w)))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_rank_and_sum_the_work():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(k, 2, port, q)) for k in range(2)]
    for p in procs:
        p.start()
    got = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r, (rank, world, local, slowest, rate) in enumerate(got):
        assert (rank, world, local) == (r, 2, r)
        assert slowest == pytest.approx(3.0)
        assert rate == pytest.approx(2 * 1000 / 3.0)


def test_single_rank_needs_no_process_group():
    assert bench.max_over_ranks(1.5, 1) == 1.5
    assert bench.whole_job_rate(500, 0.25, 1) == 2000.0
