"""The N > 1 path of bench.py on CPU: world_size-2 gloo ranks, each timing its own replica; the
whole-job throughput is world * steps over the slowest rank's time, the same on every rank."""
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


def _rank(rank: int, world: int, port: int, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    value, sec = bench.replica_throughput(1.0 + rank, 10, world, "cpu")
    out[rank] = (value, sec)
    dist.destroy_process_group()


def test_replica_throughput_two_ranks():
    world = 2
    with mp.get_context("spawn").Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(world, _free_port(), out), nprocs=world, join=True)
        res = dict(out)
    for r in range(world):
        assert res[r][1] == pytest.approx(2.0)            # the slower rank's seconds
        assert res[r][0] == pytest.approx(world * 10 / 2.0)


def test_replica_throughput_one_rank():
    import bench
    assert bench.replica_throughput(0.5, 20, 1, "cpu") == (40.0, 0.5)
