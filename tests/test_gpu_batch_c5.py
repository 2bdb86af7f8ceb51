"""The 64-view batched training workload at full size, in the launch
configuration the benchmark times: 2,000,000 Gaussians, 64 seeded views of
uneven resolution (W ~ U{320..1920}, H ~ U{240..1080}; about 19 global tile
bits, a three-pass tile partition at 8-bit digits), the batched training
step with 16x16 tiles (separate forward / residual / backward calls, whose
results the fused and persistent variants reproduce bit for bit).

- images: 64 sampled tiles (the two densest and six seeded tiles of 8
  views spread over the batch) against the FP64 oracle, at the image bar;
- four views bit-identical to rendering them alone;
- gradients: every 100th Gaussian (20,000) over all 64 views, summed over
  the views, against the oracle's summed FP64 gradient (relative L2 per
  tensor <= 1e-3).
The oracle runs in spawned host processes (one view each)."""
import multiprocessing as mp
import os

import numpy as np
import pytest

from helpers import IMAGE_ATOL, c5_target, compare_image, oracle_grad_of_view, oracle_tiles_of_view
from paper_2602_03207_gb300 import synthetic as S

pytestmark = pytest.mark.gpu

NAMES = ("means", "log_scales", "quats", "opacity_logits", "sh")


def _pool():
    return mp.get_context("spawn").Pool(max(1, min(16, os.cpu_count() or 1)))


def _renderer(scene_dev, n, cams, digit_bits):
    from paper_2602_03207_gb300 import autotune, batch
    k = autotune.measure_capacity(scene_dev, cams, 16, digit_bits)
    cap = min((1 << 31) - 1, int(k * 1.1) + 4096)
    return batch.BatchRenderer(n, cams, tile=16, digit_bits=digit_bits, key_capacity=cap)


def test_full_batch_images_against_oracle_and_single_views():
    import torch
    from paper_2602_03207_gb300 import render
    scene, cams = S.batch_scene(), S.batch_views()
    n = scene["means"].shape[0]
    dev = render.scene_to_device(scene)
    b = _renderer(dev, n, cams, 8)
    assert b.end_bit - 31 >= 17  # the partition takes three passes of at most 8 bits
    tgt = b.pack([torch.as_tensor(c5_target(c, v), device="cuda") for v, c in enumerate(cams)])
    b.step(dev, tgt)
    b.check_status()
    torch.cuda.synchronize()
    images = [im.cpu().numpy() for im in b.images()]
    ranges = b.ranges.cpu().numpy().view(np.uint32)
    t_final = b.t_final.cpu().numpy()
    n_contrib = b.n_contrib.cpu().numpy()
    # tiles to check: two densest + six seeded per view, 8 views
    jobs = []
    rng = np.random.default_rng(91)
    for v in range(0, 64, 8):
        a, z = b.tile_off[v], b.tile_off[v + 1]
        counts = (ranges[a:z, 1] - ranges[a:z, 0]).astype(np.int64)
        dense = np.argsort(-counts, kind="stable")[:2]
        rest = rng.choice(z - a, 6, replace=False)
        jobs.append((v, [int(t) for t in np.unique(np.concatenate([dense, rest]))]))
    with _pool() as pool:
        res = pool.map(oracle_tiles_of_view, jobs)
    n_tiles = 0
    for (v, tiles), (_, crops) in zip(jobs, res):
        cam = cams[v]
        tx = (cam["width"] + 15) // 16
        tf = t_final[b.pix_off[v]:b.pix_off[v + 1]].reshape(cam["height"], cam["width"])
        for t, ref in zip(tiles, crops):
            y0, x0 = (t // tx) * 16, (t % tx) * 16
            g = {"image": images[v][y0:y0 + 16, x0:x0 + 16].astype(np.float64),
                 "t_final": tf[y0:y0 + 16, x0:x0 + 16].astype(np.float64)}
            st = compare_image(g, ref, atol=IMAGE_ATOL)
            assert st["n_bad"] == 0, (v, t, st)
            n_tiles += 1
    assert n_tiles >= 64
    # four views rendered alone: bit-identical
    for v in (0, 21, 42, 63):
        c = cams[v]
        r = render.Renderer(n, c["width"], c["height"], tile=16, digit_bits=8, key_capacity=3 * n)
        img = r.forward(dev, c)
        r.check_status()
        torch.cuda.synchronize()
        np.testing.assert_array_equal(images[v], img.cpu().numpy())
        a, z = b.pix_off[v], b.pix_off[v + 1]
        np.testing.assert_array_equal(t_final[a:z], r.t_final.reshape(-1).cpu().numpy())
        np.testing.assert_array_equal(n_contrib[a:z], r.n_contrib.reshape(-1).cpu().numpy())
        del r


def test_full_batch_gradients_on_a_subsample_against_oracle():
    import torch
    from paper_2602_03207_gb300 import render
    stride = 100
    scene = {k: np.ascontiguousarray(a[::stride]) for k, a in S.batch_scene().items()}
    cams = S.batch_views()
    n = scene["means"].shape[0]
    dev = render.scene_to_device(scene)
    b = _renderer(dev, n, cams, 8)
    tgt = b.pack([torch.as_tensor(c5_target(c, v), device="cuda") for v, c in enumerate(cams)])
    g = {k: v.cpu().numpy().astype(np.float64) for k, v in b.step(dev, tgt).items()}
    b.check_status()
    with _pool() as pool:
        per_view = pool.map(oracle_grad_of_view, [(v, stride) for v in range(len(cams))])
    for k in NAMES:
        ref = sum(p[k] for p in per_view).reshape(g[k].shape)
        e = np.linalg.norm((g[k] - ref).ravel()) / max(np.linalg.norm(ref.ravel()), 1e-12)
        assert e <= 1e-3, (k, e)
