"""The benchmark's N > 1 path on CPU: two gloo ranks, each an independent
replica, agree on the max-over-ranks time and report the whole-job value."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    my_ms = 10.0 + 5.0 * rank  # rank 1 is the slow one
    mx = bench.max_over_ranks(torch, dist, my_ms, world, "cpu")
    value = bench.whole_job_gbs(step_bytes=10 ** 9, steps=4, world=world, max_ms=mx)
    q.put((rank, mx, value))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_max_time_and_weak_scaling_value():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, mx, value in res:
        assert mx == 15.0
        assert value == pytest.approx(2 * 10 ** 9 * 4 / 0.015 / 1e9)


def test_single_rank_passthrough():
    assert bench.max_over_ranks(torch, None, 7.0, 1, "cpu") == 7.0
    assert bench.whole_job_gbs(10 ** 9, 2, 1, 1000.0) == pytest.approx(2.0)
