#!/usr/bin/env python
"""Benchmark of the 3DGS render path on GB300: one step = one full frame
(ws_preprocess -> ws_cull -> ws_sort -> ws_rasterize) of the 1,000,000-
Gaussian 1920x1080 workload, cycling over its 8 orbit poses.

Prints ONE JSON line (rank 0). `--impl reference` times the FP64 CPU oracle
on the same workload instead. With torchrun (N > 1) every rank renders its
own frames (frames are independent: weak scaling, no collective in the data
path); the time is the max over ranks.

Inputs are synthetic (seeded cluster scene standing in for the paper's
trained captures) and larger than L2 (the scene is 236 MB).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOADS = {
    "hd": {"desc": "1,000,000 Gaussians, 1920x1080, SH3, 8 orbit poses", "n": 1_000_000},
    "uhd": {"desc": "6,000,000 Gaussians, 3840x2160, SH3, 8 orbit poses", "n": 6_000_000},
}
METRIC = "1080p frames/s at 1M splats"
METRICS = {"hd": METRIC, "uhd": "2160p frames/s at 6M splats"}
# DRAM bytes (read + write) per launch from one ncu capture of the current
# kernel (k_blend on the 1080p frame; k_blend_bwd and k_train on the 720p
# training step; the captures' summaries are kept under profiles/); to be
# reset to None whenever that kernel changes.
KERNEL_TRAFFIC = {("k_blend", 16): 51_944_448 + 11_329_280, ("k_blend_bwd", 16): 49_844_992 + 1_542_912,
                  ("k_train", 16): 43_082_752 + 4_845_312}
# k_blend_bwd_batch: DRAM bytes per (tile, splat) pair from one capture of
# the first 8 of the 64 views (a case small enough to capture), per tile size.
BATCH_BWD_TRAFFIC_PER_PAIR = {16: (3_824_162_000 + 986_591_232) / 17_334_892}
# k_train_batch (the fused pass on one block per (view, tile)): the same, from
# a capture of the same 8 views.
BATCH_TRAIN_TRAFFIC_PER_PAIR = {16: (5_528_209_000 + 1_125_041_000) / 17_334_892}
STAGES = ("preprocess", "cull", "sort", "rasterize")


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return {"hbm_gbs": float(p["hbm_gbs"]), "sm_max_mhz": float(p.get("sm_max_mhz", 2070.0)),
                "source": "measured"}
    except Exception:
        return {"hbm_gbs": 6800.0, "sm_max_mhz": 2070.0, "source": "fallback"}


def workload(name):
    from paper_2602_03207_gb300 import synthetic as S
    if name == "hd":
        return S.hd_scene(), [S.hd_camera(k) for k in range(8)]
    return S.uhd_scene(), [S.uhd_camera(k) for k in range(8)]


# --------------------------------------------------------------- clocks

class ClockSampler:
    """nvidia-smi clock/throttle sampling during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        self.lines = []
        if self.proc is not None:
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except Exception:
                self.proc.kill()
                out = ""
            self.lines = [l for l in out.splitlines() if l.strip()]

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in getattr(self, "lines", []):
            f = [x.strip() for x in l.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# --------------------------------------------------------- algorithmic work

def preprocess_bytes(n_all, n_opacity_ok, n_visible):
    """Bytes the pre-processing must move: logit + centre for every Gaussian
    (16 B) and depth + tile count out (8 B); scales + quaternion (28 B) for
    those past the opacity test; SH (192 B) in and centre/conic/colour/
    opacity/rect (52 B) out for the visible ones."""
    return 24 * n_all + 28 * n_opacity_ok + 244 * n_visible


def cull_bytes(n_all, keys):
    """Two reads of the tile counts, rect + depth of every Gaussian, offsets
    out, and one 8-byte key + 4-byte value per pair."""
    return (4 + 4 + 12 + 4) * n_all + 12 * keys


def sort_bytes(keys, passes):
    """Per LSD pass: histogram read of the keys (8 B) + scatter read and
    write of key and value (24 B)."""
    return 32 * keys * passes


def seg_partition_passes(end_bit):
    """Passes of the segmented sort's partition over bits [31, end_bit)."""
    return max(1, math.ceil((end_bit - 31) / 8))


def seg_sort_bytes(keys, end_bit):
    """Segmented sort: the partition's LSD passes (32 B per key each), the
    bounds kernel's read of the keys (8 B) and the local sort's read and
    write of key and value (24 B)."""
    return sort_bytes(keys, seg_partition_passes(end_bit)) + 32 * keys


def seg_sort_launches(end_bit):
    return 3 * seg_partition_passes(end_bit) + 2


def blend_work(fetched, width, height, tile):
    """Evaluations the blend must make: for every (tile, splat) pair, the
    tile's pixel centres inside the splat's opacity-aware extent box; and the
    composited pairs (alpha >= 1/255) among them are counted by sampling."""
    mean = fetched["mean2d"]
    conic = fetched["conic"].astype(np.float64)
    op = fetched["opacity"].astype(np.float64)
    keys, vals = fetched["sorted_keys"], fetched["sorted_vals"]
    tiles = (keys >> np.uint64(31)).astype(np.int64)
    g = vals.astype(np.int64)
    tx = (width + tile - 1) // tile
    a, b, c = conic[g, 0], conic[g, 1], conic[g, 2]
    det = a * c - b * b
    qc = np.maximum(0.0, 2.0 * np.log(255.0 * op[g]))
    ex, ey = np.sqrt(qc * c / det), np.sqrt(qc * a / det)
    ox, oy = (tiles % tx) * tile, (tiles // tx) * tile
    tw, th = np.minimum(tile, width - ox), np.minimum(tile, height - oy)  # edge tiles
    mx, my = mean[g, 0] - ox, mean[g, 1] - oy
    # pixel centres k + 1/2 with |k + 1/2 - m| <= e, k in [0, tw)
    wx = np.minimum(np.floor(mx + ex - 0.5), tw - 1) - np.maximum(np.ceil(mx - ex - 0.5), 0) + 1
    wy = np.minimum(np.floor(my + ey - 0.5), th - 1) - np.maximum(np.ceil(my - ey - 0.5), 0) + 1
    return float(np.sum(np.maximum(wx, 0) * np.maximum(wy, 0)))


# ------------------------------------------------------- multi-rank helpers

def rank_pose(rank, step, n_poses=8):
    """Pose rendered by `rank` at `step`: ranks start at different poses and
    each renders its own frames (no frame is shared, no collective)."""
    return (rank * 3 + step) % n_poses


def max_over_ranks(seconds, dist=None, device=None):
    """Slowest rank's time (the job's time); identity for one process."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(seconds)
    import torch
    t = torch.tensor([float(seconds)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank, world, seconds):
    """Units all ranks processed per second of the slowest rank."""
    return units_per_rank * world / seconds


def regions_needed(first_region_s, min_total_s, max_regions):
    """How many timed regions of the same K steps make the timed work last at
    least min_total_s (so the clock sampler sees the GPU under load)."""
    if first_region_s <= 0:
        return max_regions
    return int(max(1, min(max_regions, math.ceil(min_total_s / first_region_s))))


def timed_regions(run_steps, steps, stream, min_total_s=1.5, max_regions=400, dist=None, device=None):
    """Times exactly `steps` steps per region: barrier + device synchronize on
    both sides, CUDA events on the launching stream around the steps. Repeats
    the region until the timed work lasts min_total_s; returns the per-region
    seconds, the slowest rank's median region (the job's time) and the count.
    run_steps(offset, steps) enqueues steps offset .. offset + steps - 1."""
    import torch

    def one(offset):
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        run_steps(offset, steps)
        b.record(stream)
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()
        return a.elapsed_time(b) / 1e3

    times = [one(0)]
    want = regions_needed(times[0], min_total_s, max_regions)
    if dist is not None:  # every rank runs the same number of regions
        import torch as _t
        w = _t.tensor([want], dtype=_t.int64, device=device)
        dist.all_reduce(w, op=dist.ReduceOp.MAX)
        want = int(w.item())
    for r in range(1, want):
        times.append(one(r * steps))
    med = statistics.median(times)
    return times, max_over_ranks(med, dist, device), len(times)


# ------------------------------------------------------------------ ours

def sort_only(dev, steps=50, digit_bits=9):
    """Sort-only throughput: the 4,194,304-key (tile, depth) array, 44 bits,
    timed with CUDA events around each ws_sort call (input copied in
    between, outside the timed span), for the segmented sort (the
    renderer's) and the full-key LSD passes; both give the same output."""
    import torch
    from paper_2602_03207_gb300 import capi, synthetic as S
    k4, v4 = S.sort_keys()
    n = k4.size
    kk = torch.from_numpy(k4.view(np.int64)).to(dev)
    vv = torch.from_numpy(v4.view(np.int32)).to(dev)
    k1, v1, k2, v2 = torch.empty_like(kk), torch.empty_like(vv), torch.empty_like(kk), torch.empty_like(vv)
    num = torch.tensor([n, 0, 0, 0], dtype=torch.int32, device=dev)
    cam = capi.camera(S.small_forward()[1])
    out = {}
    for variant, flags in (("segmented", capi.WS_CFG_SORT_SEGMENTED), ("lsd", 0)):
        cfg = capi.config(digit_bits=digit_bits, flags=flags)
        ws = torch.zeros(capi.ws_workspace_bytes(0, n, cam, cfg), dtype=torch.uint8, device=dev)
        ts = []
        for it in range(steps + 5):
            k1.copy_(kk)
            v1.copy_(vv)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            capi.ws_sort(num, n, 0, 44, k1, v1, k2, v2, cfg, ws)
            b.record()
            torch.cuda.synchronize()
            if it >= 5:
                ts.append(a.elapsed_time(b))
        ts.sort()
        med = ts[len(ts) // 2] * 1e-3
        alg = seg_sort_bytes(n, 44) if flags else sort_bytes(n, math.ceil(44 / digit_bits))
        out[variant] = {"median_ms": round(med * 1e3, 4), "gkeys_s": round(n / med / 1e9, 3),
                        "achieved_gbs": round(alg / med / 1e9, 1)}
        del ws
    best = out["segmented"]
    return {"keys": n, "key_bits": 44, "variant": "segmented", "digit_bits": digit_bits,
            "median_ms": best["median_ms"], "gkeys_s": best["gkeys_s"], "achieved_gbs": best["achieved_gbs"],
            "lsd": out["lsd"]}


def ablation_table(scene, cams, tile, digit_bits, dev, frames=40, variants=None):
    """§4.4 / Table 5 style: per-stage times (CUDA events), pairs and peak
    device memory for the full pipeline and each ablation (-CULL: no viewport
    AABB culling; -RADIUS: opacity-independent box; -OPACITY: no sigma < 1/255
    culling). Every variant renders the same image; only the work differs."""
    import torch
    from paper_2602_03207_gb300 import capi, render
    n = scene["means"].shape[0]
    W, H = cams[0]["width"], cams[0]["height"]
    if variants is None:
        variants = {"full": 0, "-cull": capi.WS_CFG_NO_AABB_CULL, "-radius": capi.WS_CFG_FIXED_RADIUS,
                    "-opacity": capi.WS_CFG_NO_OPACITY_CULL}
    out = {}
    for name, flags in variants.items():
        # the cull's scan counts every pair even past the capacity
        probe = render.Renderer(n, W, H, tile=tile, digit_bits=digit_bits, key_capacity=4096, flags=flags,
                                device=dev)
        kmax = 0
        for cam in cams:
            probe.forward(scene, cam)
            kmax = max(kmax, probe.total_pairs())
        del probe
        torch.cuda.empty_cache()
        torch.cuda.reset_peak_memory_stats(dev)
        base_mem = torch.cuda.memory_allocated(dev)
        cap = int(math.ceil(kmax * 1.15 / 4096) * 4096)
        r = render.Renderer(n, W, H, tile=tile, digit_bits=digit_bits, key_capacity=cap, flags=flags, device=dev)
        for i in range(3):
            r.forward(scene, cams[i % len(cams)])
        torch.cuda.synchronize()
        ev = [[torch.cuda.Event(enable_timing=True) for _ in range(5)] for _ in range(frames)]
        pairs = 0
        for i in range(frames):
            cam = capi.camera(cams[i % len(cams)])
            e = ev[i]
            e[0].record()
            r.preprocess(scene, cam)
            e[1].record()
            r.cull(cam)
            e[2].record()
            r.sort()
            e[3].record()
            r.rasterize(cam)
            e[4].record()
        torch.cuda.synchronize()
        r.check_status()
        st = {s: sum(e[j].elapsed_time(e[j + 1]) for e in ev) / frames for j, s in enumerate(STAGES)}
        for cam in cams:
            r.forward(scene, cam)
            torch.cuda.synchronize()
            pairs += r.key_count()
        out[name] = {"stages_ms": {k: round(v, 4) for k, v in st.items()}, "total_ms": round(sum(st.values()), 4),
                     "mean_pairs": int(pairs / len(cams)),
                     "peak_frame_bytes": int(torch.cuda.max_memory_allocated(dev) - base_mem)}
        del r
        torch.cuda.empty_cache()
    return out


def packed_variant(scene, cams, tile, digit_bits, key_capacity, dev, steps=1000):
    """The packed-record variant (§3.2: RGBA8 colour + opacity, binary16
    ellipse axes) on the same frames: frames/s timed like the headline (no
    events between stages), plus per-stage times from a separate run."""
    import torch
    from paper_2602_03207_gb300 import capi, render
    n = scene["means"].shape[0]
    W, H = cams[0]["width"], cams[0]["height"]
    r = render.Renderer(n, W, H, tile=tile, digit_bits=digit_bits, key_capacity=key_capacity, device=dev,
                        packed=True)
    ccams = [capi.camera(c) for c in cams]
    for i in range(10):
        r.forward(scene, cams[i % len(cams)])
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for i in range(steps):
        cam = ccams[i % len(cams)]
        r.preprocess(scene, cam)
        r.cull(cam)
        r.sort()
        r.rasterize(cam)
    b.record()
    torch.cuda.synchronize()
    r.check_status()
    ms = a.elapsed_time(b) / steps
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(5)] for _ in range(200)]
    for i in range(200):
        cam = ccams[i % len(cams)]
        e = ev[i]
        e[0].record()
        r.preprocess(scene, cam)
        e[1].record()
        r.cull(cam)
        e[2].record()
        r.sort()
        e[3].record()
        r.rasterize(cam)
        e[4].record()
    torch.cuda.synchronize()
    st = {s: sum(e[j].elapsed_time(e[j + 1]) for e in ev) / 200 for j, s in enumerate(STAGES)}
    del r
    torch.cuda.empty_cache()
    return {"value": round(1e3 / ms, 2), "unit": "frames/s", "ms_per_step": round(ms, 4), "steps": steps,
            "stages_ms": {k: round(v, 4) for k, v in st.items()},
            "record_bytes_per_splat": {"packed": 20, "float": 44}}


def paper_design(scene, cams, tile, digit_bits, dev, steps=500):
    """The paper's own design in CUDA (ws_render_quads after ws_preprocess:
    global 32-bit depth sort in four 8-bit passes, opacity-sized quads,
    back-to-front "over") on the same frames, timed like the headline."""
    import torch
    from paper_2602_03207_gb300 import render
    n = scene["means"].shape[0]
    W, H = cams[0]["width"], cams[0]["height"]
    r = render.Renderer(n, W, H, tile=tile, digit_bits=digit_bits, key_capacity=min((1 << 31) - 1, 6 * n),
                        device=dev)
    pairs = 0
    for cam in cams:
        r.forward_quads(scene, cam)
        torch.cuda.synchronize()
        r.check_quads_status()
        pairs += r.key_count()
    for i in range(5):
        r.forward_quads(scene, cams[i % len(cams)])
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for i in range(steps):
        r.forward_quads(scene, cams[i % len(cams)])
    b.record()
    torch.cuda.synchronize()
    r.check_quads_status()
    ms = a.elapsed_time(b) / steps
    del r
    torch.cuda.empty_cache()
    return {"value": round(1e3 / ms, 2), "unit": "frames/s", "ms_per_step": round(ms, 4), "steps": steps,
            "mean_pairs_per_frame": int(pairs / len(cams)),
            "design": "global 32-bit depth sort (4 x 8-bit passes) + quads binned to tiles in depth order + "
                      "back-to-front over"}


def run_ours(args):
    import torch
    import torch.distributed as dist
    from paper_2602_03207_gb300 import capi, render
    if args.workload == "batch":
        return run_batch(args)
    if args.workload == "train":
        return run_train(args)

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    scene_np, cams = workload(args.workload)
    W, H = cams[0]["width"], cams[0]["height"]
    n = scene_np["means"].shape[0]
    scene = render.scene_to_device(scene_np, dev)

    # Key capacity from one frame per pose (a renderer keeps its capacity
    # from frame to frame), rounded up with 15% headroom.
    probe = render.Renderer(n, W, H, tile=args.tile, digit_bits=args.digit_bits, key_capacity=8 * n,
                            device=dev)
    kmax = 0
    for cam in cams:
        probe.forward(scene, cam)
        probe.check_status()
        kmax = max(kmax, probe.key_count())
    del probe
    cap = int(math.ceil(kmax * 1.15 / 4096) * 4096)
    r = render.Renderer(n, W, H, tile=args.tile, digit_bits=args.digit_bits, key_capacity=cap, device=dev)
    stream = torch.cuda.current_stream(dev)
    passes = math.ceil(r.end_bit / args.digit_bits)

    # warm-up
    for i in range(args.warmup):
        r.forward(scene, cams[rank_pose(rank, i)])
    r.check_status()
    # preprocess 1, cull 3, segmented sort (3 per partition pass + bounds +
    # local), rasterize: the blend, plus the tile-range scan unless the sort
    # wrote the ranges (ws_sort_tiles)
    ranges_given = bool(r.raster_cfg.flags & capi.WS_CFG_RANGES_GIVEN)
    launches_per_frame = 1 + 3 + seg_sort_launches(r.end_bit) + (1 if ranges_given else 2)

    ccams = [capi.camera(c) for c in cams]

    def frames_from(offset, k):
        for i in range(offset, offset + k):
            cam = ccams[rank_pose(rank, i)]
            r.preprocess(scene, cam)
            r.cull(cam)
            r.sort()
            r.rasterize(cam)

    # Timed regions: K frames back to back on one stream, CUDA events only
    # around the K frames (an event between stages would stop each stage's
    # first kernel from launching early under programmatic dependent launch),
    # barrier + synchronize on both sides; the region is repeated until the
    # timed work lasts --min-timed-s, and the median region is the time.
    with ClockSampler(local) as clk:
        region_s, elapsed, regions = timed_regions(frames_from, args.steps, stream, args.min_timed_s,
                                                   dist=dist if world > 1 else None, device=dev)
    r.check_status()
    frames = args.steps * world
    value = whole_job_rate(args.steps, world, elapsed)
    timing = {"regions": regions, "steps_per_region": args.steps, "statistic": "median region (max over ranks)",
              "region_ms": {"min": round(min(region_s) * 1e3, 4), "median": round(statistics.median(region_s) * 1e3, 4),
                            "max": round(max(region_s) * 1e3, 4)}}

    # Per-stage times from a separate run with an event between stages.
    stage_steps = min(args.steps, 400)
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(5)] for _ in range(stage_steps)]
    for i in range(stage_steps):
        cam = ccams[rank_pose(rank, i)]
        e = ev[i]
        e[0].record(stream)
        r.preprocess(scene, cam)
        e[1].record(stream)
        r.cull(cam)
        e[2].record(stream)
        r.sort()
        e[3].record(stream)
        r.rasterize(cam)
        e[4].record(stream)
    torch.cuda.synchronize()
    r.check_status()
    per = {s: [e[j].elapsed_time(e[j + 1]) for e in ev] for j, s in enumerate(STAGES)}
    stage_ms = {s: sum(v) / stage_steps for s, v in per.items()}
    stage_p99 = {s: float(np.percentile(v, 99)) for s, v in per.items()}

    # end to end through the C ABI (ws_render_frame_host, driven by
    # render.FramePipeline): every frame copies its scene from pinned host
    # memory and its image back to pinned host memory inside the call; two
    # slots on two streams, so frame i+1's upload overlaps frame i's render
    # and read-back
    e2e = None
    if not args.no_e2e:
        host = {k: torch.from_numpy(np.ascontiguousarray(scene_np[k])).pin_memory() for k in render.SCENE_KEYS}
        himg = [torch.empty((H, W, 3), dtype=torch.float32).pin_memory() for _ in range(2)]
        h2d = sum(v.numel() * 4 for v in host.values())
        d2h = himg[0].numel() * 4
        pipe = render.FramePipeline(n, W, H, tile=args.tile, digit_bits=args.digit_bits, key_capacity=cap,
                                    device=dev)
        k2 = max(3, min(args.steps, 200))
        for i in range(4):
            pipe.submit(host, cams[i % 8], himg[i % 2])
        pipe.synchronize()
        if world > 1:
            dist.barrier()
        main = torch.cuda.current_stream(dev)
        # three regions of k2 frames, each bracketed by a barrier and events;
        # the median region is the time (as for the device-resident value)
        e2e_s = []
        for _ in range(3):
            if world > 1:
                dist.barrier()
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(main)
            for st in pipe.streams():
                st.wait_stream(main)
            for i in range(k2):
                pipe.submit(host, cams[rank_pose(rank, i)], himg[i % 2])
            for st in pipe.streams():
                main.wait_stream(st)
            b.record(main)
            pipe.synchronize()
            e2e_s.append(max_over_ranks(a.elapsed_time(b) / 1e3, dist if world > 1 else None, dev))
        t2 = statistics.median(e2e_s)
        del pipe
        e2e = {"value": whole_job_rate(k2, world, t2), "unit": "frames/s", "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": d2h, "steps": k2,
               "regions_ms": [round(x * 1e3, 3) for x in e2e_s], "statistic": "median region",
               "link": link_bandwidth(host, himg[0], dev),
               "api": "C ABI ws_render_frame_host per frame (host scene -> device, the four stages, image -> "
                      "host), two slots on two streams: frame i+1's upload overlaps frame i's render"}

    result = None
    if rank == 0:
        result = summarize(args, r, scene, cams, stage_ms, elapsed, value, frames, e2e, clk.summary(),
                           launches_per_frame * args.steps, passes, world)
        result["timing"] = timing
        result["stages_p99_ms"] = {k: round(v, 4) for k, v in stage_p99.items()}
        if world == 1 and args.workload == "hd":
            del r, scene
            extra_workloads(args, dev, result)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()
    return result


def link_bandwidth(host, himg, dev, reps=10):
    """Plain copies of one frame's bytes over the host-device link (the scene
    to the device, the image back), GB/s: the ceiling of the end-to-end rate."""
    import torch
    dsc = {k: torch.empty_like(v, device=dev) for k, v in host.items()}
    dimg = torch.empty_like(himg, device=dev)
    s = torch.cuda.Stream(dev)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    with torch.cuda.stream(s):
        for rep in range(reps + 1):
            if rep == 1:
                ev[0].record(s)
            for k, v in host.items():
                dsc[k].copy_(v, non_blocking=True)
        ev[1].record(s)
        for _ in range(reps):
            himg.copy_(dimg, non_blocking=True)
        ev[2].record(s)
    torch.cuda.synchronize(dev)
    h2d = sum(v.numel() * v.element_size() for v in host.values()) * reps
    d2h = himg.numel() * himg.element_size() * reps
    return {"h2d_gbs": round(h2d / (ev[0].elapsed_time(ev[1]) / 1e3) / 1e9, 1),
            "d2h_gbs": round(d2h / (ev[1].elapsed_time(ev[2]) / 1e3) / 1e9, 1),
            "note": "plain pinned copies of the frame's scene and image, timed on their own"}


def frame_config(args, world):
    """The workload's configuration, identical in both arms of the benchmark."""
    scene_mb = 236 * WORKLOADS[args.workload]["n"] // 1_000_000
    return {"workload": WORKLOADS[args.workload]["desc"], "tile": args.tile, "digit_bits": args.digit_bits,
            "l2": f"inputs larger than L2 ({scene_mb} MB scene per frame)",
            "parallelism": f"replicas x{world} (independent frames)"}


def summarize(args, r, scene, cams, stage_ms, elapsed, value, frames, e2e, clocks, launches, passes, world):
    import torch
    peaks = load_peaks()
    n = r.n
    # per-pose counts for the algorithmic bytes (average over the 8 poses)
    tot = {"opok": 0, "vis": 0, "keys": 0, "evals": 0.0}
    logits = scene["opacity_logits"].double()
    n_opok = int((logits >= -math.log(254.0)).sum().item())
    for k in range(8):
        r.forward(scene, cams[k])
        torch.cuda.synchronize()
        vis = int((r.tiles_touched[:n] != 0).sum().item())
        kk = r.key_count()
        tot["vis"] += vis
        tot["keys"] += kk
        tot["opok"] += n_opok
        if k == 0:
            f = {"mean2d": (r.mean2d[:n, :2].double() + r.mean2d[:n, 2:].double()).cpu().numpy(),
                 "conic": r.conic[:n].cpu().numpy(), "opacity": r.opacity[:n].cpu().numpy(),
                 "sorted_keys": r.sorted_keys[:kk].cpu().numpy().view(np.uint64),
                 "sorted_vals": r.sorted_vals[:kk].cpu().numpy().view(np.uint32)}
            tot["evals0"] = blend_work(f, r.width, r.height, r.tile)
            tot["keys0"] = kk
    vis, opok, keys = tot["vis"] / 8, tot["opok"] / 8, tot["keys"] / 8
    b_pre = preprocess_bytes(n, opok, vis)
    b_cull = cull_bytes(n, keys)
    b_sort = seg_sort_bytes(keys, r.end_bit)
    stages = {}
    for s, b in (("preprocess", b_pre), ("cull", b_cull), ("sort", b_sort)):
        ms = stage_ms[s]
        gbs = b / (ms * 1e-3) / 1e9
        stages[s] = {"ms": round(ms, 4), "bound": "hbm", "alg_bytes": int(b), "achieved_gbs": round(gbs, 1),
                     "frac": round(gbs / peaks["hbm_gbs"], 4)}
    # blend: FP32 pipe. Per evaluated pair the kernel issues ~10 FP32
    # instructions to reach the 1/255 test and ~6 more when it composites;
    # algorithmic evaluations = pixel centres inside each pair's extent box.
    # Units: pixel centres inside a pair's extent box (pose 0, scaled to the
    # mean pair count). FLOPs: 11 per evaluation to reach the 1/255 test
    # (offsets, quadratic form, scale by opacity) + 8 to composite for the
    # pi/4 of them inside the ellipse the box bounds.
    evals = tot["evals0"] * (keys / max(tot["keys0"], 1))
    flops = fwd_flops(evals)
    ms = stage_ms["rasterize"]
    sm_count = torch.cuda.get_device_properties(0).multi_processor_count
    peak_tflops = sm_count * 128 * 2 * peaks["sm_max_mhz"] * 1e6 / 1e12
    ach = flops / (ms * 1e-3) / 1e12
    # the SFU side: one ex2 per evaluation against 16 SFU results per clock per SM
    sfu_peak = sm_count * 16 * peaks["sm_max_mhz"] * 1e6
    sfu_rate = evals / (ms * 1e-3)
    stages["rasterize"] = {"ms": round(ms, 4), "bound": "alu", "alg_evals": int(evals),
                           "achieved_tflops": round(ach, 3), "peak_tflops": round(peak_tflops, 2),
                           "frac": round(ach / peak_tflops, 4),
                           "sfu": {"achieved_gex2_s": round(sfu_rate / 1e9, 1),
                                   "peak_gex2_s": round(sfu_peak / 1e9, 1), "frac": round(sfu_rate / sfu_peak, 4)}}
    # The dominant single kernel of a frame is k_blend (largest share of the
    # ncu launch list). Its timed span is the ws_rasterize call, which also
    # holds the two small tile-range kernels, so the fraction is conservative.
    d = stages["rasterize"]
    roof = {"kernel": "k_blend<%d> (timed span: ws_rasterize)" % r.tile, "bound": "alu",
            "achieved": d["achieved_tflops"], "peak": d["peak_tflops"], "unit": "TFLOP/s", "frac": d["frac"],
            "traffic": KERNEL_TRAFFIC.get(("k_blend", r.tile)) if args.workload == "hd" else None,
            "peak_source": "derived: SMs x 128 FP32 lanes x 2 x max SM clock (no measured FP32 peak)"}
    out = {
        "metric": METRICS.get(args.workload, METRIC), "value": round(value, 2), "unit": "frames/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(elapsed / args.steps * 1e3, 4),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic (seeded 64-cluster scene standing in for the paper's trained captures)",
        "config": frame_config(args, world),
        "frame_stats": {"key_capacity": r.key_capacity, "mean_pairs_per_frame": int(keys),
                        "mean_visible": int(vis)},
        "stages_ms": {s: round(stage_ms[s], 4) for s in STAGES},
        "stages_note": "per-stage CUDA events from a separate run of the same frames with an event "
                       "between stages; the timed run has none",
        "stages": stages,
        "roofline": roof,
        "e2e": e2e,
        "gpu_launches": launches,
        "clocks": clocks,
    }
    out["sort_only"] = sort_only(r.image.device, digit_bits=args.digit_bits)
    out["paper_design"] = paper_design(scene, cams, r.tile, args.digit_bits, r.image.device,
                                       steps=min(args.steps, 500))
    out["packed_variant"] = packed_variant(scene, cams, r.tile, args.digit_bits, r.key_capacity, r.image.device,
                                           steps=min(args.steps, 1000))
    if not args.no_ablation:
        out["ablation"] = ablation_table(scene, cams, r.tile, args.digit_bits, r.image.device,
                                         frames=40 if args.workload == "hd" else 16)
    if not args.no_cpu and world == 1:
        out["cpu_baseline"] = cpu_baseline(args)
    return out


def extra_workloads(args, dev, out):
    """The other two measurements the metric names, on the same GPU in the same
    run: training steps (720p/500k fwd + bwd) and the 64-view batched step
    against 64 plain per-view steps; plus the 2160p/6M per-stage and
    peak-memory table with and without culling. Frees the frame's buffers
    first."""
    import torch
    torch.cuda.empty_cache()
    if not args.no_train:
        out["train"] = train_block(args, dev, min_timed_s=min(1.0, args.min_timed_s))
        torch.cuda.empty_cache()
    if not args.no_batch:
        out["batch"] = batch_block(args, dev)
        torch.cuda.empty_cache()
    if not args.no_uhd:
        out["uhd_stages"] = uhd_block(args, dev)
        torch.cuda.empty_cache()


def _oracle_worker(job):
    """One host process of the all-cores oracle run: renders its poses of
    the workload and returns the wall-clock span of the rendering."""
    name, poses = job
    import oracle
    scene_np, cams = workload(name)
    t0 = time.time()
    for k in poses:
        oracle.render(scene_np, cams[k])
    return t0, time.time()


def cpu_baseline(args, frames=2):
    """The FP64 oracle as it stands, over whole frames of the same workload
    (bounded): single-threaded (`frames` frames), and as one process per
    host core (up to 16; spawned, one pose each) for the all-cores rate."""
    import multiprocessing as mp
    import oracle
    scene_np, cams = workload(args.workload)
    oracle.build()
    t = time.perf_counter()
    for k in range(frames):
        oracle.render(scene_np, cams[k])
    dt = time.perf_counter() - t
    out = {"value": round(frames / dt, 4), "unit": "frames/s", "cores": 1, "kind": "oracle",
           "sample": f"{frames} full frames (poses 0..{frames - 1}) of the same workload, FP64 C oracle"}
    procs = max(1, min(16, os.cpu_count() or 1))
    if procs > 1:
        jobs = [(args.workload, [k % len(cams)]) for k in range(procs)]
        with mp.get_context("spawn").Pool(procs) as pool:
            spans = pool.map(_oracle_worker, jobs)
        wall = max(e for _, e in spans) - min(s for s, _ in spans)
        out["all_cores"] = {"value": round(procs / wall, 4), "unit": "frames/s", "cores": procs,
                            "sample": f"{procs} processes, one full frame each (poses mod 8), rate = frames / "
                                      f"(last end - first start of the rendering)"}
    return out


# ------------------------------------------------------------ training steps

BWD_FLOPS_TEST = 11.0      # per evaluation: offsets, quadratic form, the 1/255 test
BWD_FLOPS_COMPOSITE = 43.0  # per composited evaluation: T before the pair, colour,
#                             alpha, conic and centre partials


def fwd_flops(evals):
    """Algorithmic FP32 work of the forward blend over `evals` evaluations:
    11 FLOPs to the 1/255 test each, 8 more for the pi/4 that composite."""
    return evals * (11.0 + 8.0 * math.pi / 4.0)


def bwd_flops(evals):
    """Algorithmic FP32 work of the backward blend over `evals` evaluations
    (pixel centres inside a pair's extent box; pi/4 of them lie in the
    ellipse the box bounds and are composited)."""
    return evals * (BWD_FLOPS_TEST + BWD_FLOPS_COMPOSITE * math.pi / 4.0)


def fp32_peak_tflops():
    import torch
    peaks = load_peaks()
    sm_count = torch.cuda.get_device_properties(0).multi_processor_count
    return sm_count * 128 * 2 * peaks["sm_max_mhz"] * 1e6 / 1e12


def _events(k):
    import torch
    return [torch.cuda.Event(enable_timing=True) for _ in range(k)]


def train_block(args, dev, min_timed_s=1.0, stage_steps=100):
    """Single-view training steps: forward + L2 residual + backward of the
    500,000-Gaussian 1280x720 scene against a U[0,1) target (the gradient
    parity workload). Timed regions of K steps as the frame metric, for the
    separate calls (ws_rasterize, ws_image_residual, ws_rasterize_backward)
    and for the fused pass (ws_render_train_l2), which gives the same bits;
    the faster is the value. Plus a per-stage split of the separate calls
    from a run with an event between stages."""
    import torch
    from paper_2602_03207_gb300 import capi, render, synthetic as S
    scene_np, cam, target = S.grad_scene()
    n = scene_np["means"].shape[0]
    scene = render.scene_to_device(scene_np, dev)
    tgt = torch.as_tensor(target, device=dev)
    d = torch.empty_like(tgt)
    r = render.Renderer(n, cam["width"], cam["height"], tile=args.tile, digit_bits=args.digit_bits,
                        key_capacity=4 * n, device=dev)
    ccam = capi.camera(cam)
    stream = torch.cuda.current_stream(dev)

    def step():
        r.preprocess(scene, ccam)
        r.cull(ccam)
        r.sort()
        r.rasterize(ccam)
        capi.ws_image_residual(tgt.numel(), r.image, tgt, d)
        r.backward(scene, cam, d)

    def step_fused():  # pre-processing, compaction, sort, then the fused pass
        r.train_step_l2(scene, cam, tgt)

    for _ in range(max(args.warmup, 3)):
        step()
        step_fused()
    torch.cuda.synchronize()
    r.check_status()
    steps = max(3, args.steps)
    timed = {}
    with ClockSampler(dev.index) as clk:
        for name, fn in (("separate", step), ("fused", step_fused)):
            timed[name] = timed_regions(lambda o, k: [fn() for _ in range(k)], steps, stream, min_timed_s)
    r.check_status()
    path = min(timed, key=lambda nm: timed[nm][1])
    region_s, t_region, regions = timed[path]
    t = t_region / steps
    # per-stage split
    names = ("preprocess", "cull", "sort", "rasterize", "residual", "backward")
    ev = [_events(len(names) + 1) for _ in range(stage_steps)]
    for e in ev:
        e[0].record(stream)
        r.preprocess(scene, ccam)
        e[1].record(stream)
        r.cull(ccam)
        e[2].record(stream)
        r.sort()
        e[3].record(stream)
        r.rasterize(ccam)
        e[4].record(stream)
        capi.ws_image_residual(tgt.numel(), r.image, tgt, d)
        e[5].record(stream)
        r.backward(scene, cam, d)
        e[6].record(stream)
    torch.cuda.synchronize()
    stage_ms = {nm: sum(e[j].elapsed_time(e[j + 1]) for e in ev) / stage_steps for j, nm in enumerate(names)}
    # the fused path's split: the same three stages, then ws_render_train_l2
    fev = [_events(2) for _ in range(stage_steps)]
    for e in fev:
        r.preprocess(scene, ccam)
        r.cull(ccam)
        r.sort()
        e[0].record(stream)
        r.train_pass_l2(scene, cam, tgt)
        e[1].record(stream)
    torch.cuda.synchronize()
    fused_ms = sum(e[0].elapsed_time(e[1]) for e in fev) / stage_steps
    kk = r.key_count()
    f = {"mean2d": (r.mean2d[:n, :2].double() + r.mean2d[:n, 2:].double()).cpu().numpy(),
         "conic": r.conic[:n].cpu().numpy(), "opacity": r.opacity[:n].cpu().numpy(),
         "sorted_keys": r.sorted_keys[:kk].cpu().numpy().view(np.uint64),
         "sorted_vals": r.sorted_vals[:kk].cpu().numpy().view(np.uint32)}
    evals = blend_work(f, r.width, r.height, r.tile)
    peak = fp32_peak_tflops()
    if path == "fused":
        ach = (fwd_flops(evals) + bwd_flops(evals)) / (fused_ms * 1e-3) / 1e12
        roof = {"kernel": f"k_train<{r.tile}> (timed span: ws_render_train_l2)", "bound": "alu",
                "alg_evals": int(evals), "achieved": round(ach, 3), "peak": round(peak, 2), "unit": "TFLOP/s",
                "frac": round(ach / peak, 4), "traffic": KERNEL_TRAFFIC.get(("k_train", r.tile)),
                "peak_source": "derived: SMs x 128 FP32 lanes x 2 x max SM clock"}
    else:
        ach = bwd_flops(evals) / (stage_ms["backward"] * 1e-3) / 1e12
        roof = {"kernel": f"k_blend_bwd<{r.tile}> (timed span: ws_rasterize_backward)", "bound": "alu",
                "alg_evals": int(evals), "achieved": round(ach, 3), "peak": round(peak, 2), "unit": "TFLOP/s",
                "frac": round(ach / peak, 4), "traffic": KERNEL_TRAFFIC.get(("k_blend_bwd", r.tile)),
                "peak_source": "derived: SMs x 128 FP32 lanes x 2 x max SM clock"}
    return {"metric": "720p fwd+bwd steps/s at 500k splats", "value": round(1.0 / t, 2), "unit": "steps/s",
            "steps": steps, "ms_per_step": round(t * 1e3, 4),
            "timing": {"regions": regions, "steps_per_region": steps, "statistic": "median region",
                       "region_ms": {"min": round(min(region_s) * 1e3, 3),
                                     "max": round(max(region_s) * 1e3, 3)}},
            "config": {"workload": "500,000 Gaussians, 1280x720, SH3, forward + L2 residual + backward",
                       "tile": args.tile, "digit_bits": args.digit_bits, "pairs": kk,
                       "path": {"separate": "ws_rasterize + ws_image_residual + ws_rasterize_backward",
                                "fused": "ws_render_train_l2"}[path]},
            "step_variants": {nm: {"ms_per_step": round(v[1] / steps * 1e3, 4), "steps_s": round(steps / v[1], 2)}
                              for nm, v in timed.items()},
            "stages_ms": {k: round(v, 4) for k, v in stage_ms.items()},
            "stages_note": "separate calls, an event between stages; the fused pass alone (ws_render_train_l2 "
                           "after the sort): " + f"{fused_ms:.4f} ms",
            "roofline": roof,
            "clocks": clk.summary()}


def batch_block(args, dev, min_timed_s=1.0, plain_min_s=0.5):
    """Batched forward + backward of the 2,000,000-Gaussian scene over 64
    seeded views (uneven resolutions 320x240 .. 1920x1080): one training step
    (forward, L2 residual, backward, gradients summed over views) replayed as
    a CUDA graph with the autotuned tile size / digit width, against the plain
    path of 64 per-view forward + backward calls (per-view gradients, not
    summed: the comparison favours the plain path)."""
    import torch
    from paper_2602_03207_gb300 import autotune, batch, capi, render, synthetic as S
    scene_np = S.batch_scene()
    cams = S.batch_views()[:max(1, args.views)]
    n = scene_np["means"].shape[0]
    V = len(cams)
    scene = render.scene_to_device(scene_np, dev)
    rng = np.random.default_rng(9)
    targets = [torch.as_tensor(rng.random((c["height"], c["width"], 3), dtype=np.float32), device=dev)
               for c in cams]
    tgt = torch.cat([t.reshape(-1) for t in targets])
    log = (lambda m: print(m, file=sys.stderr, flush=True))
    if args.no_autotune:
        k = autotune.measure_capacity(scene, cams, args.tile, args.digit_bits)
        best = {"tile": args.tile, "digit_bits": args.digit_bits,
                "key_capacity": min((1 << 31) - 1, int(math.ceil(k * 1.1 / 4096) * 4096) + 4096),
                "table": None, "cached": None}
    else:
        best = autotune.tune(scene, cams, tgt, log=log)
    b = batch.BatchRenderer(n, cams, tile=best["tile"], digit_bits=best["digit_bits"],
                            key_capacity=best["key_capacity"], device=dev)
    stream = torch.cuda.current_stream(dev)
    steps = max(1, min(args.steps, 5))
    # The separate calls, the fused single pass on one block per (view, tile)
    # and the fused pass as one persistent grid give the same bits; each is
    # captured as a CUDA graph and timed the same way, and the fastest is the
    # value (the tuner's tile and digit width are timed on the separate calls).
    paths = [("separate", b)]
    if not args.no_variants:
        for name, persistent in (("fused_grid", False), ("fused_persistent", True)):
            paths.append((name, batch.BatchRenderer(n, cams, tile=best["tile"], digit_bits=best["digit_bits"],
                                                    key_capacity=best["key_capacity"], device=dev, fused=True,
                                                    persistent=persistent)))
    timed = {}
    with ClockSampler(dev.index) as clk:
        for name, bb in paths:
            g = bb.capture(scene, tgt)
            for _ in range(max(args.warmup, 3)):
                g.replay()
            torch.cuda.synchronize()
            timed[name] = timed_regions(lambda o, k: [g.replay() for _ in range(k)], steps, stream, min_timed_s,
                                        max_regions=50)
            bb.check_status()
            del g
    del bb
    path = min(timed, key=lambda nm: timed[nm][1])
    region_s, t_region, regions = timed[path]
    t_batch = t_region / steps
    pairs = b.key_count()
    variants = {nm: {"ms_per_step": round(v[1] / steps * 1e3, 3), "views_s": round(V / (v[1] / steps), 2)}
                for nm, v in timed.items()}
    bf = dict(paths)[path] if path != "separate" else None  # kept for the fused pass's own span
    paths = None
    torch.cuda.empty_cache()
    # per-stage split of the batched step (eager launches, an event between stages)
    names = ("preprocess", "cull", "sort", "rasterize", "residual", "backward")
    reps = 5
    ev = [_events(len(names) + 1) for _ in range(reps)]
    for e in ev:
        e[0].record(stream)
        b.preprocess(scene)
        e[1].record(stream)
        b.cull()
        e[2].record(stream)
        b.sort()
        e[3].record(stream)
        b.rasterize()
        e[4].record(stream)
        b.residual(tgt)
        e[5].record(stream)
        b.backward(scene, b.d_image)
        e[6].record(stream)
    torch.cuda.synchronize()
    b.check_status()
    stage_ms = {nm: sum(e[j].elapsed_time(e[j + 1]) for e in ev) / reps for j, nm in enumerate(names)}
    fused_ms = None
    if bf is not None:  # the fused pass alone, after the same three stages
        fev = [_events(2) for _ in range(reps)]
        for e in fev:
            bf.preprocess(scene)
            bf.cull()
            bf.sort()
            e[0].record(stream)
            bf.train_pass(scene, tgt)
            e[1].record(stream)
        torch.cuda.synchronize()
        bf.check_status()
        fused_ms = sum(e[0].elapsed_time(e[1]) for e in fev) / reps
        del bf
        torch.cuda.empty_cache()
    # algorithmic evaluations of the backward blend, summed over views
    evals = 0.0
    kk = b.key_count()
    sk = b.sorted_keys[:kk].cpu().numpy().view(np.uint64)
    sv = b.sorted_vals[:kk].cpu().numpy().view(np.uint32)
    gt = (sk >> np.uint64(31)).astype(np.int64)
    for v, c in enumerate(cams):
        lo, hi = np.searchsorted(gt, [b.tile_off[v], b.tile_off[v + 1]])
        a0, a1 = v * n, (v + 1) * n
        f = {"mean2d": (b.mean2d[a0:a1, :2].double() + b.mean2d[a0:a1, 2:].double()).cpu().numpy(),
             "conic": b.conic[a0:a1].cpu().numpy(), "opacity": b.opacity[a0:a1].cpu().numpy(),
             "sorted_keys": ((gt[lo:hi] - b.tile_off[v]).astype(np.uint64) << np.uint64(31)),
             "sorted_vals": sv[lo:hi]}
        evals += blend_work(f, c["width"], c["height"], b.tile)
    peak = fp32_peak_tflops()
    if fused_ms is None:
        ach = bwd_flops(evals) / (stage_ms["backward"] * 1e-3) / 1e12
        roof = {"kernel": f"k_blend_bwd_batch<{best['tile']}> (timed span: ws_rasterize_backward_batch)",
                "traffic": (round(BATCH_BWD_TRAFFIC_PER_PAIR[best["tile"]] * pairs)
                            if best["tile"] in BATCH_BWD_TRAFFIC_PER_PAIR else None)}
    else:
        ach = (fwd_flops(evals) + bwd_flops(evals)) / (fused_ms * 1e-3) / 1e12
        roof = {"kernel": f"k_train_batch<{best['tile']}> (timed span: ws_render_train_l2_batch, "
                          f"{'persistent grid' if path == 'fused_persistent' else 'one block per item'})",
                "traffic": (round(BATCH_TRAIN_TRAFFIC_PER_PAIR[best["tile"]] * pairs)
                            if best["tile"] in BATCH_TRAIN_TRAFFIC_PER_PAIR and path == "fused_grid" else None)}
    roof.update({"bound": "alu", "alg_evals": int(evals), "achieved": round(ach, 3), "peak": round(peak, 2),
                 "unit": "TFLOP/s", "frac": round(ach / peak, 4),
                 "traffic_note": "DRAM bytes per pair of an ncu capture of the 8-view batch (17,334,892 pairs), "
                                 "times this step's pairs",
                 "peak_source": "derived: SMs x 128 FP32 lanes x 2 x max SM clock"})
    out = {
        "metric": "batched fwd+bwd views/s", "value": round(V / t_batch, 2), "unit": "views/s",
        "steps": steps, "ms_per_step": round(t_batch * 1e3, 3),
        "timing": {"regions": regions, "steps_per_region": steps, "statistic": "median region",
                   "region_ms": {"min": round(min(region_s) * 1e3, 3), "max": round(max(region_s) * 1e3, 3)}},
        "config": {"workload": f"2,000,000 Gaussians x {V} views 320x240..1920x1080, fwd + L2 residual + bwd",
                   "tile": best["tile"], "digit_bits": best["digit_bits"], "pairs": pairs,
                   "path": {"separate": "ws_rasterize_batch + ws_image_residual + ws_rasterize_backward_batch",
                            "fused_grid": "ws_render_train_l2_batch, one block per (view, tile)",
                            "fused_persistent": "ws_render_train_l2_batch, persistent grid"}[path],
                   "autotune": best.get("table"), "autotune_cached": best.get("cached")},
        "stages_ms": {k: round(v, 3) for k, v in stage_ms.items()},
        "stages_note": "separate calls, eager launches with an event between stages"
                       + (f"; the fused pass alone (after the sort): {fused_ms:.3f} ms" if fused_ms else "")
                       + "; each timed step is one CUDA-graph replay",
        "step_variants": variants,
        "step_variants_note": "the separate forward / residual / backward calls, the fused single pass per "
                              "(view, tile) and its persistent grid give the same results; the fastest is the value",
        "roofline": roof,
        "clocks": clk.summary(),
    }
    if args.no_plain:
        return out
    del b
    torch.cuda.empty_cache()
    # plain path: one renderer per view, forward + residual + backward per view
    plain = []
    for c, t in zip(cams, targets):
        probe = render.Renderer(n, c["width"], c["height"], tile=16, digit_bits=9, key_capacity=3 * n, device=dev)
        probe.forward(scene, c)
        probe.check_status()
        cap = int(math.ceil(probe.key_count() * 1.1 / 4096) * 4096) + 4096
        del probe
        r = render.Renderer(n, c["width"], c["height"], tile=16, digit_bits=9, key_capacity=cap, device=dev)
        plain.append((r, c, capi.camera(c), t, torch.empty_like(t)))
    torch.cuda.empty_cache()

    def plain_step():
        for r, c, cc, t, d in plain:
            r.preprocess(scene, cc)
            r.cull(cc)
            r.sort()
            r.rasterize(cc)
            capi.ws_image_residual(t.numel(), r.image, t, d)
            r.backward(scene, c, d)

    for _ in range(2):
        plain_step()
    torch.cuda.synchronize()
    p_region, t_plain_region, p_regions = timed_regions(lambda o, k: [plain_step() for _ in range(k)], 1, stream,
                                                        plain_min_s, max_regions=20)
    for r, *_ in plain:
        r.check_status()
    t_plain = t_plain_region
    out.update({
        "plain": {"value": round(V / t_plain, 2), "unit": "views/s", "ms_per_step": round(t_plain * 1e3, 3),
                  "regions": p_regions,
                  "note": "64 per-view forward + residual + backward calls, per-view gradients not summed"},
        "speedup_vs_plain": round(t_plain / t_batch, 3),
    })
    return out


def uhd_block(args, dev, frames=16):
    """The 3840x2160 / 6,000,000-Gaussian workload: per-stage times and peak
    device memory of a frame over the 8 orbit poses, for the full pipeline,
    each of the three ablations, and both culls off at once (no sigma < 1/255
    cull and no viewport test)."""
    import torch
    from paper_2602_03207_gb300 import capi, render
    scene_np, cams = workload("uhd")
    scene = render.scene_to_device(scene_np, dev)
    tab = ablation_table(scene, cams, args.tile, args.digit_bits, dev, frames=frames,
                         variants={"full": 0, "-cull": capi.WS_CFG_NO_AABB_CULL,
                                   "-radius": capi.WS_CFG_FIXED_RADIUS, "-opacity": capi.WS_CFG_NO_OPACITY_CULL,
                                   "no-cull": capi.WS_CFG_NO_OPACITY_CULL | capi.WS_CFG_NO_AABB_CULL})
    del scene
    torch.cuda.empty_cache()
    return {"workload": WORKLOADS["uhd"]["desc"], "frames_per_variant": frames, "variants": tab,
            "note": "CUDA events between stages; peak = device bytes the frame's buffers hold"}


def run_train(args):
    import torch
    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", "0")))
    torch.cuda.set_device(dev)
    out = train_block(args, dev, min_timed_s=min(1.0, args.min_timed_s))
    out.update({"n_gpus": 1, "warmup": args.warmup, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f32", "data": "synthetic (seeded cluster scene, U[0,1) target)"})
    return out


def run_batch(args):
    import torch
    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", "0")))
    torch.cuda.set_device(dev)
    out = batch_block(args, dev)
    out.update({"n_gpus": 1, "warmup": max(args.warmup, 3), "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f32",
                "data": "synthetic (seeded 64-cluster scene, 64 orbit views, random U[0,1) targets)"})
    return out


# ------------------------------------------------------------- reference

_REF = {}


def _ref_init(name):
    """Worker set-up of the reference arm: the workload's scene and cameras,
    generated once per process (outside the timed span)."""
    import oracle
    _REF["scene"], _REF["cams"] = workload(name)
    oracle.lib()


def _ref_frame(k):
    """One full frame of the reference arm (pose k mod 8) by the FP64 oracle;
    returns a checksum so no image travels between processes."""
    import oracle
    img = oracle.render(_REF["scene"], _REF["cams"][k % len(_REF["cams"])])["image"]
    return float(img.sum())


def run_reference(args):
    """The FP64 oracle, as it stands, timed on the host cores on the same
    workload: every step renders one full frame (all Gaussians, full image,
    pose = step mod 8); the steps are spread over one process per host core
    (up to 16), each process single-threaded. Rank 0 alone runs it."""
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return None
    if args.workload not in WORKLOADS:
        return {"impl": "reference", "unavailable": f"the oracle arm times the frame workloads "
                                                      f"({', '.join(sorted(WORKLOADS))}), not '{args.workload}'"}
    import multiprocessing as mp
    import oracle
    oracle.build()
    procs = max(1, min(16, os.cpu_count() or 1, args.steps))
    with mp.get_context("spawn").Pool(procs, initializer=_ref_init, initargs=(args.workload,)) as pool:
        pool.map(_ref_frame, range(args.warmup), chunksize=1)
        t = time.perf_counter()
        pool.map(_ref_frame, range(args.steps), chunksize=1)
        dt = time.perf_counter() - t
    value = args.steps / dt
    return {"impl": "reference", "metric": METRICS.get(args.workload, METRIC), "value": round(value, 4),
            "unit": "frames/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(dt / args.steps * 1e3, 3), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded 64-cluster scene standing in for "
                                                        "the paper's trained captures)",
            "config": frame_config(args, world),
            "cpu_baseline": {"value": round(value, 4), "unit": "frames/s", "cores": procs, "kind": "oracle",
                             "sample": f"each step: one full frame of the workload (all Gaussians, full image); "
                                       f"steps spread over {procs} single-threaded processes"},
            "e2e": {"value": round(value, 4), "unit": "frames/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="hd", choices=sorted(WORKLOADS) + ["batch", "train"])
    ap.add_argument("--tile", type=int, default=16)
    ap.add_argument("--digit-bits", type=int, default=9)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-ablation", action="store_true")
    ap.add_argument("--no-autotune", action="store_true", help="batch: use --tile / --digit-bits as given")
    ap.add_argument("--no-plain", action="store_true", help="batch: skip the per-view comparison")
    ap.add_argument("--no-variants", action="store_true", help="batch: skip the fused single-pass variants")
    ap.add_argument("--views", type=int, default=64, help="batch: the first N of the 64 seeded views")
    ap.add_argument("--no-train", action="store_true", help="skip the training-step measurement")
    ap.add_argument("--no-batch", action="store_true", help="skip the batched-views measurement")
    ap.add_argument("--no-uhd", action="store_true", help="skip the 2160p/6M per-stage table")
    ap.add_argument("--min-timed-s", type=float, default=1.5,
                    help="repeat the K-step timed region until the timed work lasts this long")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    res = run_reference(args) if args.impl == "reference" else run_ours(args)
    if res is not None:
        print(json.dumps(res), flush=True)


if __name__ == "__main__":
    main()
