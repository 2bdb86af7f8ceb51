"""Views of a batch sharded across ranks, on CPU with gloo (world size 2):
each rank sums its views' gradients (the FP64 oracle stands in for the GPU
renderer) and the ranks combine them in a fixed rank order. The result must
equal the single-process sum over all views (to FP64 rounding), be the same
on both ranks, and be the same on a rerun."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2602_03207_gb300 import shard


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _views():
    from paper_2602_03207_gb300 import synthetic as S
    sizes = [(40, 30), (24, 36), (48, 20), (32, 32), (20, 28), (36, 24)]
    return [S.look_at_camera((3.0 * np.cos(a), 3.0 * np.sin(a), 0.7), (0, 0, 0), w, h, f=40.0)
            for a, (w, h) in zip(np.linspace(0.0, 5.0, len(sizes)), sizes)]


def _scene():
    from paper_2602_03207_gb300 import synthetic as S
    return S.uniform_scene(48, seed=61, log_scale_mean=-2.2, log_scale_std=0.3)


def _grads(views):
    """Oracle gradient of 1/2 ||C - target||^2 summed over the given views, in view order."""
    import oracle
    scene, cams = _scene(), _views()
    total = None
    for v in views:
        t = np.random.default_rng(70 + v).random((cams[v]["height"], cams[v]["width"], 3)).astype(np.float32)
        g = oracle.loss_grad(scene, cams[v], t)["grads"]
        g = {k: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)) for k, a in g.items()}
        total = g if total is None else {k: total[k] + g[k] for k in g}
    return total


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        pixels = [c["width"] * c["height"] for c in _views()]
        a = shard.sharded_step(_grads, pixels, dist)
        b = shard.sharded_step(_grads, pixels, dist)
        q.put((rank, {k: v.numpy() for k, v in a.items()}, {k: v.numpy() for k, v in b.items()}))
    finally:
        dist.destroy_process_group()


def test_shard_views_contiguous_balanced_and_complete():
    pix = [1200, 864, 960, 1024, 560, 864]
    for world in (1, 2, 3, 6):
        blocks = shard.shard_views(pix, world)
        assert [v for b in blocks for v in b] == list(range(len(pix)))
        assert all(len(b) >= 1 for b in blocks)
    b2 = shard.shard_views(pix, 2)
    assert abs(sum(pix[v] for v in b2[0]) - sum(pix[v] for v in b2[1])) <= max(pix)
    big = [1] * 64
    assert [len(b) for b in shard.shard_views(big, 8)] == [8] * 8


def test_two_ranks_sum_their_shards_in_fixed_order():
    import oracle
    oracle.build()
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted((q.get(timeout=300) for _ in range(world)), key=lambda x: x[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    ref = _grads(range(len(_views())))
    for _, a, b in res:
        for k in ref:
            np.testing.assert_array_equal(a[k], b[k])          # rerun: same bits
            np.testing.assert_array_equal(a[k], res[0][1][k])  # every rank: same bits
            np.testing.assert_allclose(a[k], ref[k].numpy(), rtol=1e-12, atol=1e-15)
