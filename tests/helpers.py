"""Shared helpers of the GPU parity tests: run the CUDA path through the C
ABI, fetch its buffers as numpy, and compare with the FP64 oracle under the
tolerances the tests state."""
import numpy as np

IMAGE_ATOL = 2e-4  # max-abs error per channel of the FP32 image vs the FP64 oracle


def gpu_frame(scene_np, cam, tile=16, digit_bits=8, key_capacity=None, flags=0):
    import torch
    from paper_2602_03207_gb300 import render
    dev = render.scene_to_device(scene_np)
    n = scene_np["means"].shape[0]
    r = render.Renderer(n, cam["width"], cam["height"], tile=tile, digit_bits=digit_bits,
                        key_capacity=key_capacity, flags=flags)
    c = capi_camera(cam)
    r.preprocess(dev, c)
    r.cull(c)
    # the sort's ping-pong overwrites the emitted list: keep a copy
    r.emitted_keys = r.keys.clone()
    r.emitted_vals = r.vals.clone()
    r.sort()
    r.rasterize(c)
    r.check_status()
    torch.cuda.synchronize()
    return r


def capi_camera(cam):
    from paper_2602_03207_gb300 import capi
    return capi.camera(cam)


def fetch(r):
    """Device buffers of a Renderer after a frame, as numpy."""
    n = r.n
    k = r.key_count()
    out = {
        "mean2d4": r.mean2d[:n].cpu().numpy(),
        "conic": r.conic[:n].cpu().numpy(),
        "depth": r.depth[:n].cpu().numpy(),
        "rgb": r.rgb[:n].cpu().numpy(),
        "opacity": r.opacity[:n].cpu().numpy(),
        "rect": r.rect[:n].cpu().numpy().view(np.uint16).astype(np.int64),
        "touched": r.tiles_touched[:n].cpu().numpy().view(np.uint32).astype(np.int64),
        "offsets": r.offsets.cpu().numpy().view(np.uint32).astype(np.int64),
        "keys": r.emitted_keys[:k].cpu().numpy().view(np.uint64),
        "vals": r.emitted_vals[:k].cpu().numpy().view(np.uint32),
        "sorted_keys": r.sorted_keys[:k].cpu().numpy().view(np.uint64),
        "sorted_vals": r.sorted_vals[:k].cpu().numpy().view(np.uint32),
        "ranges": r.ranges.cpu().numpy().view(np.uint32).astype(np.int64),
        "image": r.image.cpu().numpy().astype(np.float64),
        "t_final": r.t_final.cpu().numpy().astype(np.float64),
        "n_contrib": r.n_contrib.cpu().numpy().view(np.uint32).astype(np.int64),
        "num_keys": k,
    }
    m = out["mean2d4"].astype(np.float64)
    out["mean2d"] = m[:, :2] + m[:, 2:]
    return out


def last_gid(g, width, height, tile):
    """Gaussian index of each pixel's last composited splat (-1: none), from
    the GPU's n_contrib, sorted values and tile ranges."""
    tx = (width + tile - 1) // tile
    v, u = np.mgrid[0:height, 0:width]
    t = (v // tile) * tx + (u // tile)
    start = g["ranges"][t, 0]
    nc = g["n_contrib"]
    res = np.full((height, width), -1, np.int64)
    ok = nc > 0
    res[ok] = g["sorted_vals"][start[ok] + nc[ok] - 1]
    return res


def compare_image(g, ref, tile_mask=None, atol=IMAGE_ATOL):
    """Every pixel matches the oracle within atol; a pixel with exactly one
    ambiguous 1/255 decision may match the oracle's alternative instead;
    pixels with two or more are counted and skipped. Returns stats."""
    img, t = g["image"], g["t_final"]
    e0 = np.abs(img - ref["image"]).max(axis=-1)
    e1 = np.abs(img - ref["alt_image"]).max(axis=-1)
    t0 = np.abs(t - ref["t_final"])
    t1 = np.abs(t - ref["alt_t_final"])
    ok_primary = (e0 <= atol) & (t0 <= atol)
    ok_alt = (e1 <= atol) & (t1 <= atol) & (ref["n_amb"] == 1)
    sel = np.ones(e0.shape, bool) if tile_mask is None else tile_mask
    multi = (ref["n_amb"] >= 2) & sel
    bad = sel & ~multi & ~(ok_primary | ok_alt)
    clean = sel & (ref["n_amb"] == 0)
    stats = {"max_err_clean": float(e0[clean].max()) if clean.any() else 0.0,
             "n_bad": int(bad.sum()), "n_amb1": int(((ref["n_amb"] == 1) & sel).sum()),
             "n_multi": int(multi.sum()), "n_pix": int(sel.sum())}
    if stats["n_bad"]:
        idx = np.argwhere(bad)[:5]
        stats["examples"] = [(tuple(i), float(e0[tuple(i)]), float(e1[tuple(i)]), int(ref["n_amb"][tuple(i)]))
                             for i in idx]
    return stats


# ---- workers for the full-size batched test (spawned processes; no GPU)

def c5_target(cam, v):
    """Seeded U[0,1) target image of view v of the batched workload."""
    return np.random.default_rng(1000 + v).random((cam["height"], cam["width"], 3)).astype(np.float32)


def oracle_tiles_of_view(job):
    """FP64 oracle image of view `v` of the 2,000,000-Gaussian batch scene
    on the listed 16x16 tiles, returned as per-tile crops."""
    import oracle
    from paper_2602_03207_gb300 import synthetic as S
    v, tiles = job
    scene, cam = S.batch_scene(), S.batch_views()[v]
    ref = oracle.render(scene, cam, tile_list=np.asarray(tiles))
    tx = (cam["width"] + 15) // 16
    out = []
    for t in tiles:
        y0, x0 = (t // tx) * 16, (t % tx) * 16
        sl = (slice(y0, y0 + 16), slice(x0, x0 + 16))
        out.append({k: ref[k][sl] for k in ("image", "alt_image", "t_final", "alt_t_final", "n_amb")})
    return v, out


def oracle_grad_of_view(job):
    """FP64 oracle gradient of view `v` for every `stride`-th Gaussian of the
    batch scene against the view's seeded target."""
    import oracle
    from paper_2602_03207_gb300 import synthetic as S
    v, stride = job
    scene = {k: np.ascontiguousarray(a[::stride]) for k, a in S.batch_scene().items()}
    cam = S.batch_views()[v]
    return oracle.loss_grad(scene, cam, c5_target(cam, v))["grads"]
