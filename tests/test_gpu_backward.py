"""GPU parity of ws_rasterize_backward against the oracle's analytic FP64
gradient of L = 1/2 ||C - target||^2 (itself pinned to FP64 central
differences in the CPU suite). Bar: per-tensor relative L2 error <= 1e-3,
and bitwise-identical gradients across repeated runs."""
import numpy as np
import pytest

import oracle
from paper_2602_03207_gb300 import synthetic as S

pytestmark = pytest.mark.gpu

NAMES = ("means", "log_scales", "quats", "opacity_logits", "sh")


def gpu_grads(scene_np, cam, target, tile=16, key_capacity=None, flags=0):
    import torch
    from paper_2602_03207_gb300 import render
    dev = render.scene_to_device(scene_np)
    n = scene_np["means"].shape[0]
    r = render.Renderer(n, cam["width"], cam["height"], tile=tile, key_capacity=key_capacity, flags=flags)
    img = r.forward(dev, cam)
    r.check_status()
    d_img = img - torch.as_tensor(target, device=img.device)
    g = r.backward(dev, cam, d_img)
    torch.cuda.synchronize()
    return {k: v.cpu().numpy().astype(np.float64) for k, v in g.items()}, img.cpu().numpy()


def rel(a, b):
    return np.linalg.norm((a - b).ravel()) / max(np.linalg.norm(b.ravel()), 1e-12)


@pytest.mark.parametrize("big", [False, True])
def test_gradients_match_oracle_small(big):
    scene, cam, target = S.gradcheck_scene()
    if big:
        scene = S.uniform_scene(64, seed=7, log_scale_mean=-2.3, log_scale_std=0.3)
    g, _ = gpu_grads(scene, cam, target)
    ref = oracle.loss_grad(scene, cam, target)["grads"]
    for k in NAMES:
        assert rel(g[k], ref[k].reshape(g[k].shape)) <= 1e-3, (k, rel(g[k], ref[k].reshape(g[k].shape)))


def test_gradients_with_a_background():
    """A non-black background enters every pair's alpha derivative through
    the colour behind it (the backward starts that colour at the background):
    the separate calls and the fused pass against the oracle's gradient."""
    import torch
    from paper_2602_03207_gb300 import render
    scene, cam, target = S.gradcheck_scene()
    cam = dict(cam, bg=(0.3, 0.6, 0.9))
    g, _ = gpu_grads(scene, cam, target)
    r = render.Renderer(64, 32, 32)
    gf = r.train_step_l2(render.scene_to_device(scene), cam, torch.as_tensor(target, device="cuda"))
    r.check_status()
    ref = oracle.loss_grad(scene, cam, target)["grads"]
    for k in NAMES:
        assert rel(g[k], ref[k].reshape(g[k].shape)) <= 1e-3, (k, rel(g[k], ref[k].reshape(g[k].shape)))
        np.testing.assert_array_equal(gf[k].cpu().numpy().astype(np.float64), g[k])


@pytest.mark.parametrize("tile", [8, 32])
def test_gradients_tile_sizes(tile):
    scene, cam = S.small_forward()
    sub = {k: v[:3000] for k, v in scene.items()}
    target = np.random.default_rng(9).random((256, 256, 3)).astype(np.float32)
    g, _ = gpu_grads(sub, cam, target, tile=tile, key_capacity=16 * 3000)
    ref = oracle.loss_grad(sub, cam, target, tile=tile)["grads"]
    for k in NAMES:
        assert rel(g[k], ref[k].reshape(g[k].shape)) <= 1e-3, k


@pytest.mark.parametrize("flags", [1, 2, 8, 11])
def test_gradients_under_ablation_flags(flags):
    """The §4.4 ablations (1: keep sigma < 1/255, 2: -CULL keeps off-screen
    boxes, 8: -RADIUS opacity-independent box) only add pairs whose alpha is
    below 1/255 at every pixel: their records are zeros, added in slot order
    to sums that start at +0, so the gradients equal the default's bit for
    bit; and they match the oracle's gradient under the same flag."""
    scene = S.uniform_scene(2000, seed=53)
    scene["opacity_logits"][:200] = -7.0
    cam = S.look_at_camera((2.2, -1.0, 0.8), (0.4, 0.0, 0.0), 96, 72)
    target = np.random.default_rng(14).random((72, 96, 3)).astype(np.float32)
    import torch
    from paper_2602_03207_gb300 import render
    g, img = gpu_grads(scene, cam, target, key_capacity=60 * 2000, flags=flags)
    base, base_img = gpu_grads(scene, cam, target, key_capacity=60 * 2000)
    np.testing.assert_array_equal(img, base_img)
    for k in NAMES:
        np.testing.assert_array_equal(g[k], base[k])
    # the fused training pass under the same flag
    r = render.Renderer(2000, 96, 72, key_capacity=60 * 2000, flags=flags)
    gf = r.train_step_l2(render.scene_to_device(scene), cam, torch.as_tensor(target, device="cuda"))
    r.check_status()
    for k in NAMES:
        np.testing.assert_array_equal(gf[k].cpu().numpy().astype(np.float64), base[k])
    ref = oracle.loss_grad(scene, cam, target, flags=flags)["grads"]
    for k in NAMES:
        assert rel(g[k], ref[k].reshape(g[k].shape)) <= 1e-3, (k, rel(g[k], ref[k].reshape(g[k].shape)))


def test_gradients_of_empty_and_fully_culled_scenes():
    """n = 0 (empty gradient arrays) and a scene whose every splat is below
    1/255 (no pair at all): the image is the background, the separate calls
    and the fused pass give all-zero gradients, as the oracle does."""
    import torch
    from paper_2602_03207_gb300 import render
    cam = dict(S.small_forward()[1])
    cam["bg"] = (0.25, 0.5, 0.75)
    target = np.random.default_rng(15).random((256, 256, 3)).astype(np.float32)
    empty = S.uniform_scene(0, seed=1)
    g, img = gpu_grads(empty, cam, target)
    np.testing.assert_array_equal(img, np.broadcast_to(np.float32(cam["bg"]), img.shape))
    assert all(g[k].size == 0 for k in NAMES)
    scene = S.uniform_scene(500, seed=2)
    scene["opacity_logits"][:] = -7.0
    g, img = gpu_grads(scene, cam, target)
    np.testing.assert_array_equal(img, np.broadcast_to(np.float32(cam["bg"]), img.shape))
    r = render.Renderer(500, 256, 256)
    gf = r.train_step_l2(render.scene_to_device(scene), cam, torch.as_tensor(target, device="cuda"))
    r.check_status()
    ref = oracle.loss_grad(scene, cam, target)["grads"]
    for k in NAMES:
        assert not np.any(g[k]) and not np.any(gf[k].cpu().numpy()), k
        assert not np.any(ref[k]), k


def test_gradients_deterministic():
    scene, cam = S.small_forward()
    target = np.random.default_rng(10).random((256, 256, 3)).astype(np.float32)
    a, _ = gpu_grads(scene, cam, target)
    b, _ = gpu_grads(scene, cam, target)
    for k in NAMES:
        np.testing.assert_array_equal(a[k], b[k])


def test_autograd_function():
    import torch
    from paper_2602_03207_gb300 import render
    scene, cam, target = S.gradcheck_scene()
    params = {k: torch.tensor(v, device="cuda", requires_grad=True) for k, v in scene.items()}
    r = render.Renderer(64, 32, 32)
    img = render.render_differentiable(params, r, cam)
    loss = 0.5 * ((img - torch.as_tensor(target, device="cuda")) ** 2).sum()
    loss.backward()
    ref = oracle.loss_grad(scene, cam, target)
    assert abs(loss.item() - ref["loss"]) <= 1e-4 * abs(ref["loss"])
    for k in NAMES:
        got = params[k].grad.cpu().numpy().astype(np.float64)
        assert rel(got, ref["grads"][k].reshape(got.shape)) <= 1e-3, k


def test_training_workload_500k():
    """500,000 Gaussians at 1280x720 against a random target (the gradient
    workload): every gradient tensor against the oracle."""
    scene, cam, target = S.grad_scene()
    g, _ = gpu_grads(scene, cam, target)
    ref = oracle.loss_grad(scene, cam, target)["grads"]
    for k in NAMES:
        e = rel(g[k], ref[k].reshape(g[k].shape))
        assert e <= 1e-3, (k, e)


def test_autograd_step_captures_in_a_cuda_graph():
    """Forward + L2 loss + backward through render_differentiable never
    synchronises the host, so the whole step captures in a CUDA graph; two
    replays give gradients bit-identical to the eager step's, and the
    capacity check afterwards finds no overflow."""
    import torch
    from paper_2602_03207_gb300 import render
    scene, cam = S.small_forward()
    sub = {k: v[:3000] for k, v in scene.items()}
    target = torch.as_tensor(np.random.default_rng(12).random((256, 256, 3)).astype(np.float32), device="cuda")
    params = {k: torch.tensor(v, device="cuda", requires_grad=True) for k, v in sub.items()}
    r = render.Renderer(3000, 256, 256, key_capacity=16 * 3000)

    def step():
        img = render.render_differentiable(params, r, cam)
        loss = 0.5 * ((img - target) ** 2).sum()
        loss.backward()
        return loss

    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):  # eager warm-up (allocates the workspace), then the reference step
        for p in params.values():
            p.grad = None
        step()
        for p in params.values():
            p.grad = None
        step()
    torch.cuda.current_stream().wait_stream(side)
    torch.cuda.synchronize()
    eager = {k: p.grad.clone() for k, p in params.items()}
    for p in params.values():
        p.grad = None
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        step()
    for _ in range(2):
        for p in params.values():
            p.grad.zero_()
        g.replay()
        torch.cuda.synchronize()
        for k, p in params.items():
            assert torch.equal(p.grad, eager[k]), k
    r.check_status()
    ref = oracle.loss_grad(sub, cam, target.cpu().numpy())["grads"]
    for k in NAMES:
        got = params[k].grad.cpu().numpy().astype(np.float64)
        assert rel(got, ref[k].reshape(got.shape)) <= 1e-3, k


@pytest.mark.parametrize("tile", [8, 16, 32])
def test_fused_train_step_equals_separate_calls(tile):
    """ws_render_train_l2 (forward, L2 residual and backward records in one
    pass per tile) gives the image, final transmittance, last-contributor
    counts and gradients of ws_rasterize + ws_image_residual +
    ws_rasterize_backward bit for bit, and the gradients match the oracle."""
    import torch
    from paper_2602_03207_gb300 import capi, render
    scene, cam = S.small_forward()
    sub = {k: v[:3000] for k, v in scene.items()}
    target = np.random.default_rng(13).random((256, 256, 3)).astype(np.float32)
    tgt = torch.as_tensor(target, device="cuda")
    dev = render.scene_to_device(sub)
    r = render.Renderer(3000, 256, 256, tile=tile, key_capacity=16 * 3000)
    img = r.forward(dev, cam)
    d = torch.empty_like(tgt)
    capi.ws_image_residual(tgt.numel(), img, tgt, d)
    ga = r.backward(dev, cam, d)
    torch.cuda.synchronize()
    a = {"image": img.cpu().numpy(), "t_final": r.t_final.cpu().numpy(), "n_contrib": r.n_contrib.cpu().numpy(),
         **{k: v.cpu().numpy() for k, v in ga.items()}}
    r2 = render.Renderer(3000, 256, 256, tile=tile, key_capacity=16 * 3000)
    gb = r2.train_step_l2(dev, cam, tgt)
    r2.check_status()
    torch.cuda.synchronize()
    b = {"image": r2.image.cpu().numpy(), "t_final": r2.t_final.cpu().numpy(),
         "n_contrib": r2.n_contrib.cpu().numpy(), **{k: v.cpu().numpy() for k, v in gb.items()}}
    for k in a:
        np.testing.assert_array_equal(b[k], a[k], err_msg=k)
    ref = oracle.loss_grad(sub, cam, target, tile=tile)["grads"]
    for k in NAMES:
        got = b[k].astype(np.float64)
        assert rel(got, ref[k].reshape(got.shape)) <= 1e-3, k


def _needles(n, seed, long_axis):
    scene = S.uniform_scene(n, seed=seed)
    rng = np.random.default_rng(seed + 1)
    ls = np.full((n, 3), -6.5)
    ls[:, 0] = rng.uniform(*long_axis, n)  # one long axis per splat
    scene["log_scales"] = ls.astype(np.float32)
    scene["opacity_logits"] = rng.normal(1.0, 1.5, n).astype(np.float32)
    return scene


@pytest.mark.parametrize("tile", [8, 16, 32])
@pytest.mark.parametrize("long_axis", [(-3.0, -1.5), (-1.2, 0.3)])
def test_ellipse_masks_drop_no_contribution(tile, long_axis):
    """The backward and the fused training pass visit only the 4x4 sub-blocks
    that a splat's ellipse meets; the forward, and every call under
    WS_CFG_BOX_MASKS, every sub-block of its bounding box. A dropped visit
    that contributes would change the result, a dropped one that does not
    leaves every bit in place. On strongly anisotropic splats in random
    orientations (short needles, and long ones that cross many tiles with
    their centres off screen): the fused pass's image, final transmittance
    and last-contributor counts equal the forward's, and the gradients of
    the backward and of the fused pass equal those under WS_CFG_BOX_MASKS,
    all bit for bit. The gradients also meet the oracle's within 1e-3,
    although these splats' 2D covariances have condition numbers up to 7e4:
    the conic derivatives are summed in each splat's axis basis (in x, y
    coordinates the long needles' log-scale gradients came out several
    times too large)."""
    import torch
    from paper_2602_03207_gb300 import capi, render
    n = 2500
    scene = _needles(n, 95, long_axis)
    cam = S.look_at_camera((2.4, -0.8, 0.7), (0.0, 0.0, 0.0), 200, 136)
    target = np.random.default_rng(96).random((136, 200, 3)).astype(np.float32)
    tgt = torch.as_tensor(target, device="cuda")
    dev = render.scene_to_device(scene)
    cap = 400 * n
    out = {}
    for name, flags in (("ellipse", 0), ("box", capi.WS_CFG_BOX_MASKS)):
        r = render.Renderer(n, 200, 136, tile=tile, key_capacity=cap, flags=flags)
        img = r.forward(dev, cam)
        fwd = {"image": img.cpu().numpy(), "t_final": r.t_final.cpu().numpy(),
               "n_contrib": r.n_contrib.cpu().numpy()}
        d = torch.empty_like(tgt)
        capi.ws_image_residual(tgt.numel(), img, tgt, d)
        gs = {k: v.cpu().numpy() for k, v in r.backward(dev, cam, d).items()}
        r.check_status()
        r2 = render.Renderer(n, 200, 136, tile=tile, key_capacity=cap, flags=flags)
        gf = {k: v.cpu().numpy() for k, v in r2.train_step_l2(dev, cam, tgt).items()}
        r2.check_status()
        fused = {"image": r2.image.cpu().numpy(), "t_final": r2.t_final.cpu().numpy(),
                 "n_contrib": r2.n_contrib.cpu().numpy()}
        for k in fwd:
            np.testing.assert_array_equal(fused[k], fwd[k], err_msg=f"{name} {k}")
        for k in NAMES:
            np.testing.assert_array_equal(gf[k], gs[k], err_msg=f"{name} {k}")
        out[name] = gs
    for k in NAMES:
        np.testing.assert_array_equal(out["ellipse"][k], out["box"][k], err_msg=k)
    ref = oracle.loss_grad(scene, cam, target, tile=tile)["grads"]
    for k in NAMES:
        got = out["ellipse"][k].astype(np.float64)
        assert rel(got, ref[k].reshape(got.shape)) <= 1e-3, (k, rel(got, ref[k].reshape(got.shape)))
