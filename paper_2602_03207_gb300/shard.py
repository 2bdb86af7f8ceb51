"""Views of a batch sharded across ranks (one process per GPU).

Views are independent units: rank r renders its contiguous block of views
(blocks balanced by pixel count) with its own BatchRenderer, and the
per-Gaussian gradients are then combined by one exchange. To keep the result
independent of how the collective schedules its reduction, every rank
gathers all ranks' partial sums and adds them in rank order, so every rank
holds the same bits, and a rerun gives the same bits again.
"""
from __future__ import annotations

import torch


def shard_views(pixels, world):
    """Contiguous blocks of view indices, one per rank, balanced by pixel
    count: the boundary between blocks r - 1 and r is placed where the
    running pixel total comes closest to r / world of the whole. Every rank
    gets at least one view when there are at least `world` views."""
    n = len(pixels)
    if world <= 0:
        raise ValueError("world must be positive")
    total = float(sum(pixels))
    bounds = [0]
    run = 0.0
    v = 0
    for r in range(1, world):
        goal = total * r / world
        while v < n and n - (v + 1) >= world - r and (
                v < bounds[-1] + 1 or abs(run + pixels[v] - goal) < abs(run - goal)):
            run += pixels[v]
            v += 1
        bounds.append(v)
    bounds.append(n)
    return [list(range(bounds[r], bounds[r + 1])) for r in range(world)]


def fixed_order_allreduce(grads, dist):
    """Sum of every rank's gradient tensors, added in rank order 0, 1, ...
    (all-gather, then a fixed-order sum), returned on every rank. grads:
    dict name -> tensor (same shapes on every rank)."""
    world = dist.get_world_size()
    if world == 1:
        return {k: grads[k] for k in sorted(grads)}
    out = {}
    for k in sorted(grads):
        t = grads[k].contiguous()
        parts = [torch.empty_like(t) for _ in range(world)]
        dist.all_gather(parts, t)
        acc = parts[0].clone()
        for p in parts[1:]:
            acc += p
        out[k] = acc
    return out


def sharded_step(grad_fn, pixels, dist):
    """One sharded training step: this rank's views (shard_views), their
    gradient summed over the rank's views by grad_fn(view_indices) (e.g. a
    BatchRenderer step), then fixed_order_allreduce."""
    rank, world = dist.get_rank(), dist.get_world_size()
    mine = shard_views(pixels, world)[rank]
    return fixed_order_allreduce(grad_fn(mine), dist)


def batch_grad_fn(scene, cams, targets, **renderer_kw):
    """grad_fn for sharded_step on a GPU: a BatchRenderer over the given views
    (targets: list of per-view (H, W, 3) device tensors) and one training step;
    the gradients summed over those views in view order."""
    from .batch import BatchRenderer

    def fn(views):
        b = BatchRenderer(scene["means"].shape[0], [cams[v] for v in views], **renderer_kw)
        g = b.step(scene, b.pack([targets[v] for v in views]))
        b.check_status()
        return {k: v.clone() for k, v in g.items()}
    return fn
