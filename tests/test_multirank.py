"""The N > 1 bench path on CPU: two gloo ranks, each timing its own replica; the job's step time
is the slowest rank's and the throughput counts every rank's points (weak scaling, no data
exchanged between replicas)."""

import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        local = [0.010, 0.025][rank]
        t = bench.max_over_ranks(local, True, "cpu")
        v = bench.replica_throughput(10 ** 6, world, t)
        out[rank] = (t, v)
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_replica():
    ctx = mp.get_context("spawn")
    manager = ctx.Manager()
    out = manager.dict()
    port = _free_port()
    mp.start_processes(_worker, args=(2, port, out), nprocs=2, join=True, start_method="spawn")
    assert out[0] == out[1]
    t, v = out[0]
    assert t == pytest.approx(0.025)
    assert v == pytest.approx(2 * 10 ** 6 / 0.025)


def test_single_process_needs_no_collective():
    import bench
    assert bench.max_over_ranks(0.5, False) == 0.5
    assert bench.replica_throughput(100, 1, 0.5) == 200.0
