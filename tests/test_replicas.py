"""The multi-GPU path runs independent replicas (one process per GPU, no
data-path collective): each rank renders its own frames of the camera path,
and the job's time is the slowest rank's. Host logic of that path, on two
gloo ranks on CPU."""
import os
import socket
import sys

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms = [12.5, 17.25][rank]
        frags = [1000.0, 2500.0][rank]
        e2e = [0.75, 0.5][rank]
        q.put((rank, bench.reduce_replicas(ms, frags, e2e, torch.device("cpu"))))
    finally:
        dist.destroy_process_group()


def test_replica_reduction_two_gloo_ranks():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    got = dict(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    # every rank sees the slowest span and the total work
    for r in range(world):
        assert got[r] == pytest.approx((17.25, 3500.0, 0.75))


def test_replica_frames_are_disjoint_and_cover_the_path():
    n = 120
    for world in (1, 2, 4, 8):
        per = n // world
        seen = [f for r in range(world) for f in bench.replica_frames(r, world, n, 0, per)]
        assert len(set(seen)) == per * world          # no two replicas draw the same view
        assert all(0 <= f < n for f in seen)
    # a replica walks the path from its own start, wrapping around
    assert bench.replica_frames(1, 2, 120, 58, 4) == [118, 119, 0, 1]
    assert bench.replica_frames(0, 1, 120, 0, 60, stride=2) == list(range(0, 120, 2))
