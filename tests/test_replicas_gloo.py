"""The N > 1 path of bench.py (replicas only) on CPU: two gloo ranks, each with its own
system and its own time; the whole-job throughput counts both ranks' planes over the slower
rank's time."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank: int, world: int, port: int, ms_per_rank, out):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        w, r, _ = bench.dist_env()
        assert (w, r) == (world, rank)
        value, t_max = bench.replica_throughput(5 * 10, ms_per_rank[rank], world, "cpu")
        out[rank] = (value, t_max)
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_replica_throughput():
    world, port = 2, _free_port()
    ms = [8.0, 10.0]                                   # rank 1 is the slower replica
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank_main, args=(world, port, ms, out), nprocs=world, join=True)
        res = dict(out)
    for rank in range(world):
        value, t_max = res[rank]
        assert t_max == pytest.approx(10.0)
        assert value == pytest.approx(2 * 50 / 0.010)   # both ranks' 50 planes over the max time


def test_single_rank_needs_no_collective():
    sys.path.insert(0, ROOT)
    import bench
    value, t_max = bench.replica_throughput(50, 10.0, 1)
    assert (value, t_max) == (pytest.approx(5000.0), 10.0)
