"""The N-GPU bench path on the host: replicas (one camera stream per rank, no data
exchange) whose job time is the slowest rank's. Two gloo ranks on the CPU check the
max-over-ranks reduction, the whole-job rate and the pose split."""
from __future__ import annotations

import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms = bench.slowest_ms(10.0 + 5.0 * rank, dist, "cpu")  # rank 1 is the slower one
    fps = bench.job_fps(20, world, ms)
    poses = [bench.rank_pose(rank, world, k, 30) for k in range(20)]
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, ms, fps, poses))


def test_two_gloo_ranks_time_by_the_slowest_and_split_the_orbit():
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, ms0, fps0, poses0), (r1, ms1, fps1, poses1) = res
    assert ms0 == ms1 == 15.0  # both ranks report the slowest rank's time
    assert fps0 == fps1 == pytest.approx(2 * 20 / 0.015)  # all ranks' frames over that time
    assert set(poses0).isdisjoint(poses1)  # interleaved poses, no shared work
    assert sorted(set(poses0) | set(poses1)) == list(range(30))


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.slowest_ms(7.5) == 7.5
    assert bench.job_fps(300, 1, 750.0) == pytest.approx(400.0)
    assert [bench.rank_pose(0, 1, k, 30) for k in (0, 29, 30)] == [0, 29, 0]
