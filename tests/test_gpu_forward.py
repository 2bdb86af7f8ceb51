"""GPU parity of the forward render path (C ABI) against the FP64 oracle.

Tolerances: cull mask, tile rectangles, depth keys, emitted pairs and the
sort permutation are bit-exact on every decision the oracle does not flag
as within float32 rounding of its threshold (flagged ones may go either
way); the image is within 2e-4 per channel (max abs) of the oracle, or of
its alternative for a pixel with one flagged 1/255 decision.
"""
import numpy as np
import pytest

import oracle
from paper_2602_03207_gb300 import synthetic as S

from helpers import IMAGE_ATOL, capi_camera, compare_image, fetch, gpu_frame, last_gid

pytestmark = pytest.mark.gpu


def _check_preprocess(g, ref, n_amb_max=None):
    p = ref["proj"]
    amb = p["amb"].astype(bool)
    vis_ref = p["touched"] > 0
    vis_gpu = g["touched"] > 0
    # depth: identical float32 for every Gaussian
    np.testing.assert_array_equal(g["depth"].view(np.uint32), p["depth"].view(np.uint32))
    # cull mask bit-exact on unambiguous decisions
    assert np.array_equal(vis_gpu[~amb], vis_ref[~amb])
    both = vis_ref & vis_gpu & ~amb
    np.testing.assert_array_equal(g["rect"][both], p["rect"][both])
    np.testing.assert_array_equal(g["touched"][both], p["touched"][both])
    # ambiguous ones: each bound within one tile of the oracle's
    a = amb & vis_ref & vis_gpu
    if a.any():
        assert np.abs(g["rect"][a] - p["rect"][a]).max() <= 1
    vv = vis_ref & vis_gpu
    np.testing.assert_allclose(g["mean2d"][vv], p["mean2d"][vv], rtol=0, atol=2e-6)
    # conic: what the blend uses is the quadratic form q = d^T Q d; its
    # relative error r over all directions d is the spectral radius of
    # Sigma'_ref (Q_gpu - Q_ref). It moves alpha = sigma exp(-q/2) by at most
    # sigma (q/2) e^{-q/2} r <= 0.37 sigma r (largest at q = 2), so r <= 5e-4
    # keeps every pixel inside the 2e-4 image bound. (FP32 inversion of an
    # elongated Sigma' loses about eps * Sigma'_xx Sigma'_yy / det: 1.6e-4 for
    # the worst of the 3.8M splats of the 4K workload.)
    cov = p["cov2d"][vv]
    dq = g["conic"][vv].astype(np.float64) - p["conic"][vv]
    S2 = np.stack([np.stack([cov[:, 0], cov[:, 1]], -1), np.stack([cov[:, 1], cov[:, 2]], -1)], -2)
    D2 = np.stack([np.stack([dq[:, 0], dq[:, 1]], -1), np.stack([dq[:, 1], dq[:, 2]], -1)], -2)
    metric = np.abs(np.linalg.eigvals(S2 @ D2)).max(-1)
    assert metric.max() <= 5e-4, metric.max()
    np.testing.assert_allclose(g["rgb"][vv], p["rgb"][vv], rtol=0, atol=2e-6)
    np.testing.assert_allclose(g["opacity"][vv], p["opacity"][vv], rtol=2e-6, atol=0)
    if n_amb_max is not None:
        assert amb.sum() <= n_amb_max


def _check_emission(g, ref):
    p = ref["proj"]
    touched_g = g["touched"]
    np.testing.assert_array_equal(np.diff(g["offsets"]), touched_g)
    same = (p["amb"] == 0) & (touched_g == p["touched"])
    kg = np.repeat(same, touched_g)
    kr = np.repeat(same, p["touched"])
    np.testing.assert_array_equal(g["keys"][kg], ref["keys"][kr])
    np.testing.assert_array_equal(g["vals"][kg], ref["vals"][kr])


def _check_sort(g):
    k, v = oracle.sort_pairs(g["keys"], g["vals"])
    np.testing.assert_array_equal(g["sorted_keys"], k)
    np.testing.assert_array_equal(g["sorted_vals"], v)


def test_small_forward_parity():
    """10,000 Gaussians, 256x256, 16x16 tiles: every stage against the oracle."""
    scene, cam = S.small_forward()
    r = gpu_frame(scene, cam)
    g = fetch(r)
    ref = oracle.render(scene, cam)
    _check_preprocess(g, ref, n_amb_max=20)
    _check_emission(g, ref)
    _check_sort(g)
    st = compare_image(g, ref)
    assert st["n_bad"] == 0, st
    assert st["max_err_clean"] <= IMAGE_ATOL
    assert st["n_multi"] <= 0.001 * st["n_pix"]
    ok = ref["n_amb"] == 0
    np.testing.assert_array_equal(last_gid(g, 256, 256, 16)[ok], ref["last_gid"][ok])


@pytest.mark.parametrize("tile", [8, 32])
def test_tile_sizes(tile):
    scene, cam = S.small_forward()
    sub = {k: v[:3000] for k, v in scene.items()}
    g = fetch(gpu_frame(sub, cam, tile=tile, key_capacity=16 * len(sub["means"])))
    ref = oracle.render(sub, cam, tile=tile)
    _check_preprocess(g, ref)
    _check_emission(g, ref)
    _check_sort(g)
    st = compare_image(g, ref)
    assert st["n_bad"] == 0, st


def test_digit_widths_give_identical_frames():
    """The sort's digit width changes the pass structure, never the result."""
    scene, cam = S.small_forward()
    imgs = []
    for bits in (4, 5, 6, 7, 8, 9, 10, 11):
        g = fetch(gpu_frame(scene, cam, digit_bits=bits))
        imgs.append((g["image"], g["sorted_keys"], g["sorted_vals"]))
    for im, k, v in imgs[1:]:
        np.testing.assert_array_equal(im, imgs[0][0])
        np.testing.assert_array_equal(k, imgs[0][1])
        np.testing.assert_array_equal(v, imgs[0][2])


def test_ragged_resolution_and_background():
    """A 100x75 image (partial tiles on two edges), a coloured background and
    a camera looking at the scene off-centre."""
    scene = S.uniform_scene(4000, seed=31)
    cam = S.look_at_camera((2.0, -2.5, 1.0), (0.2, 0.1, 0.0), 100, 75, bg=(0.2, 0.5, 0.9))
    g = fetch(gpu_frame(scene, cam))
    ref = oracle.render(scene, cam)
    _check_preprocess(g, ref)
    _check_sort(g)
    st = compare_image(g, ref)
    assert st["n_bad"] == 0, st


def test_culled_entries_are_written_as_zeros():
    """Every output entry is written: a culled Gaussian's splat record (centre,
    conic, opacity, colour, axis word) and rect are zeros, whatever the
    buffers held before; a visible one's axis word t = tan(theta / 2) gives
    the major axis of the oracle's 2D covariance."""
    import torch
    from paper_2602_03207_gb300 import render
    scene, cam = S.small_forward()
    scene = dict(scene)
    scene["opacity_logits"] = scene["opacity_logits"].copy()
    scene["opacity_logits"][::3] = -7.0  # below 1/255: culled
    n = scene["means"].shape[0]
    r = render.Renderer(n, cam["width"], cam["height"])
    r.splats.fill_(float("nan"))
    r.rect.fill_(-1)
    r.preprocess(render.scene_to_device(scene), capi_camera(cam))
    torch.cuda.synchronize()
    g = {"mean2d4": r.mean2d[:n].cpu().numpy(), "conic": r.conic[:n].cpu().numpy(),
         "rgb": r.rgb[:n].cpu().numpy(), "opacity": r.opacity[:n].cpu().numpy(),
         "rect": r.rect[:n].cpu().numpy().view(np.uint16),
         "touched": r.tiles_touched[:n].cpu().numpy().view(np.uint32)}
    culled = g["touched"] == 0
    assert 0 < culled.sum() < n
    for k in ("mean2d4", "conic", "rgb", "opacity", "rect"):
        np.testing.assert_array_equal(g[k][culled], 0)
        assert np.isfinite(g[k][~culled].astype(np.float64)).all(), k
    t = r.splats[:n, 11].cpu().numpy().astype(np.float64)
    np.testing.assert_array_equal(t[culled], 0)
    assert (np.abs(t[~culled]) <= 1.0).all()
    # the axis (theta modulo pi) against the oracle's covariance: compare
    # (cos 2 theta, sin 2 theta), which the eigenvector's sign leaves alone,
    # where the eigenvalues differ enough to fix the axis
    ref = oracle.preprocess(scene, cam)
    cov = ref["cov2d"][~culled]
    h, b2 = 0.5 * (cov[:, 0] - cov[:, 2]), cov[:, 1]
    d = np.hypot(h, b2)
    gap = d / (0.5 * (cov[:, 0] + cov[:, 2]))
    th = 2.0 * np.arctan(t[~culled])
    ok = gap > 1e-3
    assert ok.sum() > 100
    # float32 covariance entries (relative error ~1e-6) turn the axis by
    # about that error over the relative eigenvalue gap
    tol = 1e-5 + 4e-6 / gap[ok]
    assert (np.abs(np.cos(2 * th) - h / d)[ok] <= tol).all()
    assert (np.abs(np.sin(2 * th) - b2 / d)[ok] <= tol).all()


def test_empty_and_fully_culled_scenes():
    """n = 0 and a scene whose every splat is below 1/255 give the background."""
    cam = dict(S.small_forward()[1])
    cam["bg"] = (0.25, 0.5, 0.75)
    scene = S.uniform_scene(0, seed=1)
    g = fetch(gpu_frame(scene, cam))
    assert g["num_keys"] == 0
    np.testing.assert_array_equal(g["image"], np.broadcast_to(np.float32(cam["bg"]), g["image"].shape))
    scene = S.uniform_scene(500, seed=2)
    scene["opacity_logits"][:] = -7.0
    g = fetch(gpu_frame(scene, cam))
    assert g["num_keys"] == 0 and (g["touched"] == 0).all()
    np.testing.assert_array_equal(g["t_final"], 1.0)


def test_single_splat_and_offscreen():
    """One splat centred on a pixel centre (C = c * min(.99, sigma)) and one
    fully outside the viewport (culled)."""
    scene = S.uniform_scene(2, seed=3)
    scene["means"][:] = [[(10.5 - 128) / 256 * 3.0, (20.5 - 128) / 256 * 3.0, 0.0], [50.0, 0.0, 0.0]]
    scene["log_scales"][:] = -4.0
    scene["opacity_logits"][:] = 0.7
    _, cam = S.small_forward()
    g = fetch(gpu_frame(scene, cam))
    ref = oracle.render(scene, cam)
    assert list(g["touched"] > 0) == [True, False]
    assert abs(g["image"][20, 10] - ref["image"][20, 10]).max() <= 1e-5
    st = compare_image(g, ref)
    assert st["n_bad"] == 0, st


def test_capacity_overflow_is_reported():
    from paper_2602_03207_gb300 import capi
    scene, cam = S.small_forward()
    with pytest.raises(capi.WsError):
        gpu_frame(scene, cam, key_capacity=1000)


def test_frames_are_bitwise_deterministic():
    scene, cam = S.small_forward()
    a = fetch(gpu_frame(scene, cam))
    b = fetch(gpu_frame(scene, cam))
    for k in ("image", "t_final", "n_contrib", "sorted_keys", "sorted_vals", "keys", "vals"):
        np.testing.assert_array_equal(a[k], b[k])


def test_hd_workload_sampled():
    """The 1,000,000-Gaussian 1920x1080 workload in the benchmark's launch
    configuration (16x16 tiles, 9-bit digits, the segmented sort writing the
    tile ranges): every Gaussian's pre-processing, the whole pair list and
    sort, and the image on 96 sampled tiles (the densest 32 plus 64 seeded
    ones) against the oracle."""
    scene = S.hd_scene()
    cam = S.hd_camera(0)
    r = gpu_frame(scene, cam, digit_bits=9)
    g = fetch(r)
    tx, ty = (1920 + 15) // 16, (1080 + 15) // 16
    counts = g["ranges"][:, 1] - g["ranges"][:, 0]
    dense = np.argsort(-counts, kind="stable")[:32]
    rng = np.random.default_rng(77)
    tiles = np.unique(np.concatenate([dense, rng.choice(tx * ty, 64, replace=False)]))
    ref = oracle.render(scene, cam, tile_list=tiles)
    _check_preprocess(g, ref, n_amb_max=int(0.005 * len(scene["means"])))
    _check_emission(g, ref)
    _check_sort(g)
    mask = np.zeros((1080, 1920), bool)
    for t in tiles:
        y0, x0 = (t // tx) * 16, (t % tx) * 16
        mask[y0:y0 + 16, x0:x0 + 16] = True
    st = compare_image(g, ref, tile_mask=mask)
    assert st["n_bad"] == 0, st
    assert st["n_multi"] <= 0.001 * st["n_pix"]


def test_uhd_workload_sampled():
    """The 6,000,000-Gaussian 3840x2160 workload (pose 3, whose densest tile
    holds 4,389 pairs: the segmented sort's global-memory path): every
    Gaussian's pre-processing, the whole pair list and sort, and the image on
    the densest 32 plus 64 seeded tiles against the oracle, in the
    benchmark's launch configuration (16x16 tiles, 9-bit digits)."""
    scene = S.uhd_scene()
    cam = S.uhd_camera(3)
    r = gpu_frame(scene, cam, digit_bits=9)
    g = fetch(r)
    tx, ty = (3840 + 15) // 16, (2160 + 15) // 16
    counts = g["ranges"][:, 1] - g["ranges"][:, 0]
    assert counts.max() > 2048
    dense = np.argsort(-counts, kind="stable")[:32]
    rng = np.random.default_rng(78)
    tiles = np.unique(np.concatenate([dense, rng.choice(tx * ty, 64, replace=False)]))
    ref = oracle.render(scene, cam, tile_list=tiles)
    _check_preprocess(g, ref, n_amb_max=int(0.005 * len(scene["means"])))
    _check_emission(g, ref)
    _check_sort(g)
    mask = np.zeros((2160, 3840), bool)
    for t in tiles:
        y0, x0 = (t // tx) * 16, (t % tx) * 16
        mask[y0:y0 + 16, x0:x0 + 16] = True
    st = compare_image(g, ref, tile_mask=mask)
    assert st["n_bad"] == 0, st
    assert st["n_multi"] <= 0.001 * st["n_pix"]


def test_lookback_sort_frame_identical():
    """A whole frame with the single-sweep look-back sort is bit-identical
    to the default wait-free sort."""
    from paper_2602_03207_gb300 import capi
    scene, cam = S.small_forward()
    a = fetch(gpu_frame(scene, cam, digit_bits=8))
    b = fetch(gpu_frame(scene, cam, digit_bits=8, flags=capi.WS_CFG_SORT_LOOKBACK))
    for k in ("image", "t_final", "n_contrib", "sorted_keys", "sorted_vals"):
        np.testing.assert_array_equal(a[k], b[k])


@pytest.mark.parametrize("flags", [1, 2, 8, 11])
def test_ablation_flags(flags):
    """§4.4 ablations (1: keep sigma < 1/255, 2: -CULL keeps off-screen
    boxes, 8: -RADIUS opacity-independent box): parity with the oracle under
    the same flag, and an image bit-identical to the default (they only add
    pairs whose alpha is below 1/255)."""
    scene = S.uniform_scene(4000, seed=52)
    scene["opacity_logits"][:300] = -7.0
    cam = S.look_at_camera((2.2, -1.0, 0.8), (0.4, 0.0, 0.0), 160, 120)
    g = fetch(gpu_frame(scene, cam, flags=flags, key_capacity=40 * 4000))
    ref = oracle.render(scene, cam, flags=flags)
    _check_preprocess(g, ref)
    _check_emission(g, ref)
    _check_sort(g)
    st = compare_image(g, ref)
    assert st["n_bad"] == 0, st
    base = fetch(gpu_frame(scene, cam, key_capacity=40 * 4000))
    np.testing.assert_array_equal(g["image"], base["image"])
    np.testing.assert_array_equal(g["t_final"], base["t_final"])
    assert g["num_keys"] > base["num_keys"]


def test_sort_variants_give_identical_frames():
    """The segmented sort (the renderer's default), the full-key passes and
    the look-back passes sort the 1M-splat 1080p pair list identically."""
    import torch
    from paper_2602_03207_gb300 import capi, render
    scene = render.scene_to_device(S.hd_scene())
    cam = S.hd_camera(1)
    out = {}
    for sort in ("segmented", "lsd", "lookback"):
        r = render.Renderer(1_000_000, 1920, 1080, digit_bits=8, key_capacity=1_400_000, sort=sort)
        r.forward(scene, cam)
        r.check_status()
        torch.cuda.synchronize()
        k = r.key_count()
        out[sort] = (r.sorted_keys[:k].cpu().numpy(), r.sorted_vals[:k].cpu().numpy(), r.image.cpu().numpy())
    for sort in ("lsd", "lookback"):
        for a, b in zip(out["segmented"], out[sort]):
            np.testing.assert_array_equal(a, b)


def test_ply_scene_renders_like_the_original(tmp_path):
    """A scene written to and read back from a 3DGS PLY file renders the
    same frame as the in-memory scene, within the oracle's bar."""
    from paper_2602_03207_gb300 import ply
    scene, cam = S.small_forward()
    path = tmp_path / "scene.ply"
    ply.save_ply(path, scene)
    loaded = ply.load_ply(path)
    a = fetch(gpu_frame(loaded, cam))
    b = fetch(gpu_frame(scene, cam))
    np.testing.assert_array_equal(a["image"], b["image"])
    st = compare_image(a, oracle.render(loaded, cam))
    assert st["n_bad"] == 0, st


def test_frame_pipeline_matches_renderer():
    """Frames from host memory through render.FramePipeline (one C-ABI
    ws_render_frame_host call per frame: the scene's upload, the four stages
    and the image's read-back; two slots, so uploads overlap renders) are
    bit-identical to Renderer frames."""
    import torch
    from paper_2602_03207_gb300 import render
    scene, _ = S.small_forward()
    cams = [S.look_at_camera((2.2 * np.cos(a), 2.2 * np.sin(a), 0.8), (0.0, 0.0, 0.0), 200, 150)
            for a in np.linspace(0, 2, 5)]
    host = {k: torch.from_numpy(np.ascontiguousarray(scene[k])).pin_memory() for k in render.SCENE_KEYS}
    outs = [torch.empty((150, 200, 3), dtype=torch.float32).pin_memory() for _ in cams]
    pipe = render.FramePipeline(scene["means"].shape[0], 200, 150, key_capacity=200_000)
    for c, o in zip(cams, outs):
        pipe.submit(host, c, o)
    pipe.synchronize()
    dev = render.scene_to_device(scene)
    r = render.Renderer(scene["means"].shape[0], 200, 150, key_capacity=200_000)
    for c, o in zip(cams, outs):
        ref = r.forward(dev, c).cpu()
        np.testing.assert_array_equal(o.numpy(), ref.numpy())


def test_screen_filling_splats():
    """A few splats whose extent spans most of the screen (hundreds of tiles
    each: the emission's binary-search path) over many small ones, with two
    dense clusters so that one tile holds more than 2,048 pairs and another
    257 to 2,048 (the segmented sort's global-memory and block paths):
    pre-processing, emission, sort and image against the oracle."""
    scene = S.uniform_scene(6000, seed=91)
    rng = np.random.default_rng(92)
    big = np.arange(12)
    scene["means"][big] = rng.uniform(-0.5, 0.5, (12, 3))
    scene["log_scales"][big] = np.log(rng.uniform(0.6, 1.5, (12, 3)))
    scene["opacity_logits"][big] = -2.0  # sigma ~ 0.12: wide, translucent
    # two dense clusters of tiny splats: ~3,000 pairs in one tile (the
    # segmented sort's global-memory path) and ~700 in another (its block path)
    for sl, centre in ((slice(100, 3100), (0.3, 0.2, 0.1)), (slice(3100, 3800), (-0.4, -0.1, 0.2))):
        k = sl.stop - sl.start
        scene["means"][sl] = np.asarray(centre) + rng.normal(0.0, 0.004, (k, 3))
        scene["log_scales"][sl] = -7.0
    cam = S.look_at_camera((2.6, -1.0, 0.9), (0.0, 0.0, 0.0), 320, 240)
    g = fetch(gpu_frame(scene, cam, key_capacity=60 * 6000))
    ref = oracle.render(scene, cam)
    assert ref["proj"]["touched"][big].max() >= 200
    counts = np.sort(ref["ranges"][:, 1] - ref["ranges"][:, 0])[::-1]
    assert counts[0] > 2048 and 256 < counts[1] <= 2048, counts[:4]
    _check_preprocess(g, ref)
    _check_emission(g, ref)
    _check_sort(g)
    st = compare_image(g, ref)
    assert st["n_bad"] == 0, st


def test_needle_splats():
    """Strongly anisotropic splats (axis ratios up to e^5, ~150:1) in random
    orientations: projection, extent, emission, sort and image against the
    oracle (the dilation bounds the 2D covariance's conditioning)."""
    scene = S.uniform_scene(3000, seed=93)
    rng = np.random.default_rng(94)
    ls = np.full((3000, 3), -6.5)
    ls[:, 0] = rng.uniform(-3.0, -1.5, 3000)  # one long axis per splat
    scene["log_scales"] = ls.astype(np.float32)
    scene["opacity_logits"] = rng.normal(1.0, 1.0, 3000).astype(np.float32)
    cam = S.look_at_camera((2.4, -0.8, 0.7), (0.0, 0.0, 0.0), 256, 192)
    g = fetch(gpu_frame(scene, cam, key_capacity=40 * 3000))
    ref = oracle.render(scene, cam)
    _check_preprocess(g, ref, n_amb_max=30)
    _check_emission(g, ref)
    _check_sort(g)
    st = compare_image(g, ref)
    assert st["n_bad"] == 0, st
    assert st["n_multi"] <= 0.001 * st["n_pix"]
