"""ws_cull_sort_tiles: the compaction fused into the first partition pass of
the segmented tile sort gives the offsets, key count, sorted pairs, tile
ranges and status of ws_cull followed by ws_sort_tiles, bit for bit; past
the key capacity it flags the frame and leaves only valid pairs."""
import numpy as np
import pytest

from paper_2602_03207_gb300 import synthetic as S

pytestmark = pytest.mark.gpu


def _frames(scene_np, cam, tile=16, digit_bits=9, key_capacity=None, flags=0):
    import torch
    from paper_2602_03207_gb300 import capi, render
    dev = render.scene_to_device(scene_np)
    n = scene_np["means"].shape[0]
    c = capi.camera(cam)
    out = []
    for fused in (False, True):
        r = render.Renderer(n, cam["width"], cam["height"], tile=tile, digit_bits=digit_bits,
                            key_capacity=key_capacity, flags=flags)
        r.preprocess(dev, c)
        if fused:
            r.cull_sort(c)
            assert getattr(r, "_fused_cull", True), "the fused call should apply"
        else:
            r.cull(c)
            r.sort()
        torch.cuda.synchronize()
        k = min(int(r.num_keys[0].item()), r.key_capacity)
        out.append({"offsets": r.offsets[:n + 1].cpu().numpy(), "num_keys": r.num_keys[:1].cpu().numpy(),
                    "keys": r.sorted_keys[:k].cpu().numpy(), "vals": r.sorted_vals[:k].cpu().numpy(),
                    "ranges": r.ranges[:r.tx * r.ty].cpu().numpy(),
                    "status": capi.ws_read_status(r.workspace, clear=False), "r": r})
    return out


def _same(a, b):
    for k in ("offsets", "num_keys", "keys", "vals", "ranges", "status"):
        np.testing.assert_array_equal(np.asarray(b[k]), np.asarray(a[k]), err_msg=k)


@pytest.mark.parametrize("case", ["hd0", "hd3", "train", "small4", "small9", "ragged"])
def test_fused_cull_sort_equals_separate_calls(case):
    """First digits of 7 (1080p), 6 (720p), 4 (256 tiles at 4-bit digits: two
    passes), 8 (256 tiles at 9-bit digits: the whole partition in the
    compaction) and 6 bits (35 tiles of a ragged 100x75 image)."""
    if case.startswith("hd"):
        scene, cam, kw = S.hd_scene(), S.hd_camera(int(case[2])), {}
    elif case == "train":
        scene, cam, _ = S.grad_scene()
        kw = {}
    elif case == "ragged":
        scene, cam = S.small_forward()
        cam = dict(cam, width=100, height=75)
        kw = {"key_capacity": 40 * len(scene["means"])}
    else:
        scene, cam = S.small_forward()
        kw = {"digit_bits": int(case[5:]), "key_capacity": 40 * len(scene["means"])}
    a, b = _frames(scene, cam, **kw)
    assert a["num_keys"][0] > 0
    _same(a, b)


def test_fused_cull_sort_rows_wider_than_the_digit_range():
    """Large splats: at 1280x720 (80-tile rows, 6-bit first digit) 719 of
    2,000 rectangles have rows wider than the 64 digits, so a row adds a full
    turn of the digits plus a run that may wrap; at 256x256 with 4-bit digits
    496 have 16-tile rows, exactly one turn. Also with the culling switched
    off (rectangles clamped into the grid)."""
    from paper_2602_03207_gb300 import capi
    scene = S.uniform_scene(2000, seed=5, log_scale_mean=-1.0, log_scale_std=0.4)
    cam = S.look_at_camera((2.4, -0.8, 0.7), (0.0, 0.0, 0.0), 1280, 720)
    for flags in (0, capi.WS_CFG_NO_AABB_CULL | capi.WS_CFG_NO_OPACITY_CULL):
        a, b = _frames(scene, cam, key_capacity=8_000_000, flags=flags)
        assert not (a["status"] & capi.WS_FLAG_CAPACITY)
        _same(a, b)
    _, cam = S.small_forward()
    scene = S.uniform_scene(3000, seed=5, log_scale_mean=-1.0, log_scale_std=0.4)
    a, b = _frames(scene, cam, digit_bits=4, key_capacity=600_000)
    assert not (a["status"] & capi.WS_FLAG_CAPACITY)
    _same(a, b)


@pytest.mark.parametrize("case", ["culled", "one_tile", "two_tiles"])
def test_fused_cull_sort_degenerate_frames(case):
    """A frame whose every splat is culled (no pairs), a 12x10 image (one
    tile) and a 30x10 image (two tiles): the fused call gives what the two
    calls give."""
    scene, cam = S.small_forward()
    scene = {k: v[:2000].copy() for k, v in scene.items()}
    if case == "culled":
        scene["opacity_logits"][:] = -7.0
    else:
        cam = dict(cam, width=12 if case == "one_tile" else 30, height=10)
    a, b = _frames(scene, cam, key_capacity=64 * 2000)
    _same(a, b)
    if case == "culled":
        assert int(a["num_keys"][0]) == 0


def test_fused_cull_sort_uhd():
    """6,000,000 Gaussians at 3840x2160: 15 tile bits, first digit 8."""
    a, b = _frames(S.uhd_scene(), S.uhd_camera(3))
    _same(a, b)


def test_fused_cull_sort_past_capacity_keeps_valid_pairs():
    """More pairs than the key capacity: the frame is flagged, the count is
    the capacity, and every stored pair names a Gaussian of the frame and a
    tile of the grid (the compaction falls back to slot order), so the
    rasterisation that follows reads only valid records."""
    import torch
    from paper_2602_03207_gb300 import capi
    scene, cam = S.small_forward()
    n = len(scene["means"])
    a, b = _frames(scene, cam, key_capacity=1024)
    for fr in (a, b):
        assert fr["status"] & capi.WS_FLAG_CAPACITY
        assert int(fr["num_keys"][0]) == 1024
        assert (fr["vals"].view(np.uint32) < n).all()
        tiles = fr["keys"].view(np.uint64) >> np.uint64(31)
        assert (tiles < fr["r"].tx * fr["r"].ty).all()
    r = b["r"]
    r.rasterize(capi.camera(cam))
    torch.cuda.synchronize()
    assert np.isfinite(r.image.cpu().numpy()).all()
