"""GPU parity of the paper's own render design in CUDA (ws_render_quads:
global 32-bit depth sort in four 8-bit passes, opacity-sized quads with the
local coordinate of E9, back-to-front "over") against the FP64 oracle, with
the float path's bar: every pixel within 2e-4, or within 2e-4 of the
oracle's alternative where exactly one 1/255 decision is ambiguous."""
import numpy as np
import pytest

import oracle
from paper_2602_03207_gb300 import synthetic as S

from helpers import compare_image, fetch, gpu_frame

pytestmark = pytest.mark.gpu


def quad_frame(scene_np, cam, tile=16, key_capacity=None, check=True):
    import torch
    from paper_2602_03207_gb300 import render
    dev = render.scene_to_device(scene_np)
    n = scene_np["means"].shape[0]
    r = render.Renderer(n, cam["width"], cam["height"], tile=tile, key_capacity=key_capacity)
    r.forward_quads(dev, cam)
    torch.cuda.synchronize()
    if check:
        r.check_quads_status()
    return {"image": r.image.cpu().numpy(), "t_final": r.t_final.cpu().numpy(), "num_keys": r.key_count(),
            "renderer": r}


def test_quads_small_forward():
    scene, cam = S.small_forward()
    g = quad_frame(scene, cam, key_capacity=80_000)
    ref = oracle.render(scene, cam)
    st = compare_image(g, ref)
    assert st["n_bad"] == 0, st


@pytest.mark.parametrize("tile", [8, 16, 32])
def test_quads_tile_sizes_ragged(tile):
    scene = S.uniform_scene(3000, seed=81)
    cam = S.look_at_camera((2.4, -1.2, 1.0), (0.3, 0.1, 0.0), 173, 101)
    g = quad_frame(scene, cam, tile=tile, key_capacity=60 * 3000)
    ref = oracle.render(scene, cam, tile=tile)
    st = compare_image(g, ref)
    assert st["n_bad"] == 0, st


def test_quads_match_tile_path_and_are_deterministic():
    """Same image as the tile path within float rounding; two runs
    bit-identical; the quad boxes bin at least as many pairs as the
    ellipse boxes."""
    scene = S.uniform_scene(4000, seed=82)
    cam = S.look_at_camera((2.2, -1.0, 0.8), (0.4, 0.0, 0.0), 160, 120)
    a = quad_frame(scene, cam, key_capacity=60 * 4000)
    b = quad_frame(scene, cam, key_capacity=60 * 4000)
    np.testing.assert_array_equal(a["image"], b["image"])
    t = fetch(gpu_frame(scene, cam, key_capacity=60 * 4000))
    assert np.abs(a["image"] - t["image"]).max() <= 2e-4
    assert a["num_keys"] >= t["num_keys"]


def test_quads_hd_sampled():
    """The 1M-splat 1080p workload: the image on 64 sampled tiles."""
    scene = S.hd_scene()
    cam = S.hd_camera(2)
    g = quad_frame(scene, cam, key_capacity=2_500_000)
    tx, ty = (1920 + 15) // 16, (1080 + 15) // 16
    rng = np.random.default_rng(83)
    tiles = np.unique(rng.choice(tx * ty, 64, replace=False))
    ref = oracle.render(scene, cam, tile_list=tiles)
    mask = np.zeros((1080, 1920), bool)
    for t in tiles:
        mask[(t // tx) * 16:(t // tx) * 16 + 16, (t % tx) * 16:(t % tx) * 16 + 16] = True
    st = compare_image(g, ref, tile_mask=mask)
    assert st["n_bad"] == 0, st


def test_quads_capacity_overflow_is_reported():
    from paper_2602_03207_gb300 import capi
    scene, cam = S.small_forward()
    g = quad_frame(scene, cam, key_capacity=1000, check=False)
    with pytest.raises(capi.WsError):
        g["renderer"].check_quads_status()


def test_quads_empty_scene():
    scene = S.uniform_scene(500, seed=84)
    scene["opacity_logits"][:] = -9.0  # all below 1/255
    cam = S.look_at_camera((2.2, -1.0, 0.8), (0.4, 0.0, 0.0), 64, 48)
    g = quad_frame(scene, cam, key_capacity=4096)
    np.testing.assert_array_equal(g["t_final"], np.ones_like(g["t_final"]))
    np.testing.assert_allclose(g["image"], np.broadcast_to(np.asarray(cam["bg"], np.float32), g["image"].shape))


def test_quads_no_gaussians():
    cam = S.look_at_camera((2.2, -1.0, 0.8), (0.4, 0.0, 0.0), 64, 48)
    empty = {k: v[:0] for k, v in S.uniform_scene(10, seed=1).items()}
    g = quad_frame(empty, cam, key_capacity=4096)
    assert g["num_keys"] == 0
    np.testing.assert_array_equal(g["t_final"], np.ones_like(g["t_final"]))
    np.testing.assert_allclose(g["image"], np.broadcast_to(np.asarray(cam["bg"], np.float32), g["image"].shape))
