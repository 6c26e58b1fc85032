"""Replicas across ranks: each rank builds its own octree from its own
stream, and the job's throughput is the total points over the slowest rank's
time. The host logic runs here as two gloo ranks on the CPU."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

import bench  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms, pts = bench.aggregate(10.0 + 5.0 * rank, 1000 * (rank + 1), dist, "cpu")
        w, _ = bench.rank_workload("uniform", 2000, rank)
        first = tuple(int(v) for v in w.points[0].tolist()[:3])
        out[rank] = (ms, pts, first)
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_aggregate_and_own_streams():
    world = 2
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_worker, args=(world, _free_port(), out), nprocs=world,
                       start_method="spawn", join=True)
    assert out[0][:2] == out[1][:2] == (15.0, 3000)  # max time, total points
    assert out[0][2] != out[1][2]  # different streams per rank


def test_single_rank_aggregate_is_identity():
    assert bench.aggregate(3.5, 42) == (3.5, 42)
