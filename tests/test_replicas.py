"""Replica aggregation of bench.py on two gloo ranks (CPU): every rank sees the
slowest rank's time, and the whole-job value counts the units of all ranks."""
import os
import socket
import sys

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    sys.path.insert(0, ROOT)
    import bench
    # rank r took (r + 1) * 100 ms for 3e9 units of its own work
    max_ms, value = bench.aggregate(100.0 * (rank + 1), 3e9, world, "cpu")
    dist.barrier()
    q.put((rank, max_ms, value))
    dist.destroy_process_group()


def test_two_rank_aggregation():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    world, port = 2, _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    out = sorted(q.get(timeout=10) for _ in range(world))
    for rank, max_ms, value in out:
        assert max_ms == pytest.approx(200.0)
        assert value == pytest.approx(2 * 3e9 / 0.2 / 1e9)   # 30 Gunits/s


def test_single_rank_is_local():
    sys.path.insert(0, ROOT)
    import bench
    max_ms, value = bench.aggregate(250.0, 1e9, 1, "cpu")
    assert max_ms == 250.0 and value == pytest.approx(4.0)
