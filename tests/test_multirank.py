"""The N > 1 path of bench.py on CPU: two gloo ranks (127.0.0.1) draw their
own data (weak scaling), the job's time is the slowest rank's (all-reduce
MAX), and the whole-job throughput counts every rank's units over it.  No
GPU: the same helpers take the NCCL group on the GPUs."""
from __future__ import annotations

import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank: int, world: int, port: int, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import bench

    dist.init_process_group("gloo", rank=rank, world_size=world)
    w, r, local = bench.dist_env()
    ms = [12.5, 20.25][rank]  # rank 1 is the slow one
    slowest = bench.max_over_ranks(dist, ms, "cpu")
    value = bench.job_throughput(w, 3 * 200_000_000, slowest)
    seed = bench.rank_seed(1234, r)
    out.put((r, w, local, slowest, value, seed))
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time_and_count_every_rank():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [x[0] for x in res] == [0, 1] and all(x[1] == 2 for x in res)
    assert all(x[3] == pytest.approx(20.25) for x in res)          # max over ranks, on every rank
    assert all(x[4] == pytest.approx(2 * 6e8 / 0.02025) for x in res)  # whole-job units / slowest time
    assert res[0][5] != res[1][5]                                    # own data per rank


def test_single_process_needs_no_group():
    import bench

    assert bench.max_over_ranks(None, 7.0, "cpu") == 7.0
    assert bench.job_throughput(1, 100, 1000.0) == pytest.approx(100.0)
