"""Multi-rank timing of bench.py (replicas): two gloo ranks on the CPU."""
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
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    secs = bench.max_over_ranks(1.0 + 0.5 * rank, dist, "cpu")
    q.put((rank, secs, bench.job_value(world, 256, 2, secs)))
    dist.destroy_process_group()


def test_two_ranks_take_the_slowest_time():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
    assert all(p.exitcode == 0 for p in procs)
    for rank, secs, value in out:
        assert secs == 1.5
        assert abs(value - 2 * 256 * 2 / 1.5) < 1e-9


def test_single_rank_is_unchanged():
    assert bench.max_over_ranks(3.25, None, "cpu") == 3.25
    assert bench.job_value(1, 256, 1, 2.0) == 128.0
