"""Multi-GPU runs of bench.py are independent replicas (one solve does not
shard): every rank solves its own seeded instance and the whole-job rate is
all ranks' iterations over the slowest rank's time.  This checks that host
logic with two gloo ranks on the CPU (no GPU needed)."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, times, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        rate, tmax = bench.replica_rate(times[rank], 300, world)
        out[rank] = (rate, tmax, bench.replica_seed(1000, rank))
    finally:
        dist.destroy_process_group()


def test_two_replicas_rate_uses_the_slowest_rank():
    world = 2
    times = [0.5, 0.8]
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(world, _free_port(), times, out), nprocs=world, join=True)
        res = dict(out)
    for r in range(world):
        rate, tmax, _ = res[r]
        assert tmax == pytest.approx(0.8)
        assert rate == pytest.approx(300 * world / 0.8)
    assert res[0][2] != res[1][2]  # each rank solves its own instance


def test_single_process_rate():
    rate, tmax = bench.replica_rate(0.25, 300, 1)
    assert tmax == 0.25 and rate == pytest.approx(1200.0)
