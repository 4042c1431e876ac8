"""Replica timing of bench.py across ranks (gloo, world size 2, CPU): the whole-job value
counts every rank's pairs over the slowest rank's time."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as tmp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    local_ms = 100.0 + 50.0 * rank          # rank 1 is slower
    slowest = bench.reduce_max(local_ms, world)
    out[rank] = (slowest, bench.replica_throughput(1280 * 720 * 128, 10, world, slowest))
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_use_the_slowest_time():
    world = 2
    port = _free_port()
    mgr = tmp.Manager()
    out = mgr.dict()
    tmp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
    assert out[0][0] == out[1][0] == 150.0
    want = 2 * 10 * 1280 * 720 * 128 / 0.150 / 1e6
    assert abs(out[0][1] - want) < 1e-6 * want


def test_single_rank_is_identity():
    import bench
    assert bench.reduce_max(12.5, 1) == 12.5
    assert bench.replica_throughput(100, 4, 1, 2000.0) == 100 * 4 / 2.0 / 1e6
