"""The N>1 path of bench.py on CPU: two gloo ranks (replicas) aggregate the
per-rank step times by their maximum and count the pairs of every rank."""
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


def _rank(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms = 100.0 if rank == 0 else 250.0  # the second replica is slower
    value, ms_max = bench.aggregate(ms, 100, world, dist)
    out[rank] = (value, ms_max)
    dist.barrier()
    dist.destroy_process_group()


def test_two_replicas_aggregate_by_slowest_rank():
    world = 2
    port = _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    for r in range(world):
        value, ms_max = res[r]
        assert ms_max == 250.0
        assert value == pytest.approx(world * 100 / 0.25)


def test_single_rank_aggregate():
    import bench
    value, ms_max = bench.aggregate(50.0, 10, 1, None)
    assert ms_max == 50.0 and value == pytest.approx(200.0)
