"""GPU parity of the packed-record variant (§3.2: RGBA8 colour + opacity,
binary16 ellipse axes, float32 centre) against the oracle with the same
packing (oracle.PACKED). Bar: each pixel within 1/255 per channel, the
precision the packed record keeps; pixels with two or more ambiguous 1/255
decisions are skipped as in the float path. Both sides round their own
float32 / float64 values to 8 bits and binary16, so a value within rounding
of a quantisation step can land one step apart; most pixels agree far more
closely than the bar, which the median check states."""
import numpy as np
import pytest

import oracle
from paper_2602_03207_gb300 import synthetic as S

from helpers import compare_image

pytestmark = pytest.mark.gpu

PACKED_ATOL = 1.0 / 255


def packed_frame(scene_np, cam, tile=16, key_capacity=None, flags=0):
    import torch
    from paper_2602_03207_gb300 import capi, render
    dev = render.scene_to_device(scene_np)
    n = scene_np["means"].shape[0]
    r = render.Renderer(n, cam["width"], cam["height"], tile=tile, key_capacity=key_capacity, flags=flags,
                        packed=True)
    r.forward(dev, cam)
    r.check_status()
    torch.cuda.synchronize()
    return {"image": r.image.cpu().numpy(), "t_final": r.t_final.cpu().numpy(),
            "n_contrib": r.n_contrib.cpu().numpy().view(np.uint32),
            "touched": r.tiles_touched[:n].cpu().numpy().view(np.uint32),
            "depth": r.depth[:n].cpu().numpy(), "mean2d": r.mean2d_p[:n].cpu().numpy(),
            "axes": r.axes[:n].cpu().numpy().view(np.uint32), "rgba": r.rgba[:n].cpu().numpy().view(np.uint32),
            "num_keys": r.key_count()}


def _decode_axes(w):
    h = w.view(np.uint16).reshape(-1, 4).view(np.float16).astype(np.float64)
    v1, v2 = h[:, 0:2], h[:, 2:4]
    sxx = v1[:, 0] ** 2 + v2[:, 0] ** 2
    sxy = v1[:, 0] * v1[:, 1] + v2[:, 0] * v2[:, 1]
    syy = v1[:, 1] ** 2 + v2[:, 1] ** 2
    return np.stack([sxx, sxy, syy], axis=1)


def _check_record(g, ref):
    p = ref["proj"]
    both = (g["touched"] > 0) & (p["touched"] > 0) & (p["amb"] == 0)
    assert both.sum() > 0.9 * (p["touched"] > 0).sum()
    np.testing.assert_array_equal(g["depth"].view(np.uint32), p["depth"].view(np.uint32))
    # RGBA8: each byte the oracle's 8-bit value, or one step from it where the
    # float value sits on a rounding boundary
    bytes_g = np.stack([(g["rgba"] >> s) & 255 for s in (0, 8, 16, 24)], axis=1)[both].astype(np.int64)
    bytes_o = np.rint(np.concatenate([p["rgb"], p["opacity"][:, None]], axis=1)[both] * 255).astype(np.int64)
    diff = np.abs(bytes_g - bytes_o)
    assert diff.max() <= 1 and (diff > 0).mean() < 1e-3, ((diff > 0).mean(), diff.max())
    np.testing.assert_allclose(g["mean2d"][both], p["mean2d"][both], rtol=0, atol=1e-3)
    # the packed axes rebuild Sigma' within binary16 precision of the oracle's
    cov = _decode_axes(g["axes"][both])
    scale = np.maximum(p["cov2d"][both][:, 0], p["cov2d"][both][:, 2])
    assert (np.abs(cov - p["cov2d"][both]).max(axis=1) / scale).max() <= 3e-3


def test_packed_small_forward():
    scene, cam = S.small_forward()
    g = packed_frame(scene, cam)
    ref = oracle.render(scene, cam, flags=oracle.PACKED)
    _check_record(g, ref)
    st = compare_image(g, ref, atol=PACKED_ATOL)
    assert st["n_bad"] == 0, st
    assert np.median(np.abs(g["image"] - ref["image"])) <= 1e-4


@pytest.mark.parametrize("tile", [8, 16, 32])
def test_packed_tile_sizes_and_ragged_frame(tile):
    scene = S.uniform_scene(3000, seed=71)
    cam = S.look_at_camera((2.4, -1.2, 1.0), (0.3, 0.1, 0.0), 173, 101)
    g = packed_frame(scene, cam, tile=tile, key_capacity=40 * 3000)
    ref = oracle.render(scene, cam, flags=oracle.PACKED, tile=tile)
    _check_record(g, ref)
    st = compare_image(g, ref, atol=PACKED_ATOL)
    assert st["n_bad"] == 0, st


def test_packed_hd_sampled():
    """The 1M-splat 1080p workload: the packed record of every visible
    Gaussian and the image on 64 sampled tiles (the densest 16 + 48)."""
    scene = S.hd_scene()
    cam = S.hd_camera(0)
    g = packed_frame(scene, cam, key_capacity=1_400_000)
    tx, ty = (1920 + 15) // 16, (1080 + 15) // 16
    rng = np.random.default_rng(79)
    ref0 = oracle.render(scene, cam, flags=oracle.PACKED, tile_list=np.array([0]))
    counts = ref0["ranges"][:, 1] - ref0["ranges"][:, 0]
    tiles = np.unique(np.concatenate([np.argsort(-counts, kind="stable")[:16], rng.choice(tx * ty, 48, replace=False)]))
    ref = oracle.render(scene, cam, flags=oracle.PACKED, tile_list=tiles)
    _check_record(g, ref)
    mask = np.zeros((1080, 1920), bool)
    for t in tiles:
        mask[(t // tx) * 16:(t // tx) * 16 + 16, (t % tx) * 16:(t % tx) * 16 + 16] = True
    st = compare_image(g, ref, tile_mask=mask, atol=PACKED_ATOL)
    assert st["n_bad"] == 0, st


def test_packed_close_to_float_path_and_deterministic():
    """Where no colour exceeds 1, the packed frame is within 1/255 of the
    float path's frame; two packed frames are bit-identical."""
    from helpers import fetch, gpu_frame
    scene = S.uniform_scene(3000, seed=72)
    scene["sh"][:, 0, :] = np.clip(scene["sh"][:, 0, :], -0.6, 0.6)
    scene["sh"][:, 1:, :] *= 0.2
    cam = S.look_at_camera((2.4, -1.2, 1.0), (0.3, 0.1, 0.0), 160, 120)
    a = packed_frame(scene, cam, key_capacity=40 * 3000)
    b = packed_frame(scene, cam, key_capacity=40 * 3000)
    np.testing.assert_array_equal(a["image"], b["image"])
    f = fetch(gpu_frame(scene, cam, key_capacity=40 * 3000))
    assert np.abs(a["image"] - f["image"]).max() <= 1.0 / 255


def test_packed_empty_and_fully_culled():
    """n = 0 and a scene whose every splat is below 1/255 both give the
    background with transmittance 1."""
    cam = S.look_at_camera((2.2, -1.0, 0.8), (0.4, 0.0, 0.0), 64, 48)
    empty = {k: v[:0] for k, v in S.uniform_scene(10, seed=1).items()}
    culled = S.uniform_scene(300, seed=2)
    culled["opacity_logits"][:] = -9.0
    for sc in (empty, culled):
        g = packed_frame(sc, cam, key_capacity=4096)
        assert g["num_keys"] == 0
        np.testing.assert_array_equal(g["t_final"], np.ones_like(g["t_final"]))
        np.testing.assert_allclose(g["image"], np.broadcast_to(np.asarray(cam["bg"], np.float32), g["image"].shape))
