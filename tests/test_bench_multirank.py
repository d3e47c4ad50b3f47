"""The multi-rank aggregation of bench.py (replicas, one process per GPU) on CPU
ranks over gloo: units add up over ranks, time is the slowest rank's."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    units, span = bench.aggregate(1000 * (rank + 1), 0.5 + rank, dist, torch, "cpu")
    q.put((rank, units, span))
    dist.destroy_process_group()


def test_aggregate_two_gloo_ranks():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    got = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for _, units, span in got:
        assert units == 3000 and span == 1.5


def test_aggregate_single_rank():
    import bench
    assert bench.aggregate(77, 0.25, None, torch, "cpu") == (77, 0.25)
