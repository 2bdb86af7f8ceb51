"""The N > 1 benchmark path on CPU: world size 2 over gloo. Frames are
independent, so each rank renders its own poses with no collective on the
data path; the only collective is the max-over-ranks of the timed span."""
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


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        local = [0.5, 0.8][rank]
        t = bench.max_over_ranks(local, dist)
        poses = [bench.rank_pose(rank, i) for i in range(8)]
        q.put((rank, t, poses))
    finally:
        dist.destroy_process_group()


def test_two_ranks_take_the_slowest_time_and_render_distinct_poses():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [t for _, t, _ in res] == [0.8, 0.8]
    # every rank cycles through all 8 poses, starting at a different one
    assert sorted(res[0][2]) == list(range(8)) and sorted(res[1][2]) == list(range(8))
    assert res[0][2][0] != res[1][2][0]
    assert bench.whole_job_rate(100, 2, 0.8) == pytest.approx(250.0)


def test_single_process_is_identity():
    assert bench.max_over_ranks(1.25, None) == 1.25
