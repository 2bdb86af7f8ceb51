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


# ------------------------------------------------------------------ ours

def run_ours(args):
    import torch
    import torch.distributed as dist
    from paper_2602_03207_gb300 import capi, render

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
    launches_per_frame = 1 + 3 + 3 * passes + 2

    # warm-up
    for i in range(args.warmup):
        r.forward(scene, cams[(rank + i) % 8])
    r.check_status()

    # stage timing events (per step, on the launching stream)
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(5)] for _ in range(args.steps)]
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        t_start = torch.cuda.Event(enable_timing=True)
        t_end = torch.cuda.Event(enable_timing=True)
        t_start.record(stream)
        for i in range(args.steps):
            cam = capi.camera(cams[(rank * 3 + i) % 8])
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
        t_end.record(stream)
        torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    elapsed = t_start.elapsed_time(t_end) / 1e3
    r.check_status()
    stage_ms = {s: 0.0 for s in STAGES}
    for e in ev:
        for j, s in enumerate(STAGES):
            stage_ms[s] += e[j].elapsed_time(e[j + 1])
    stage_ms = {s: v / args.steps for s, v in stage_ms.items()}
    if world > 1:
        t = torch.tensor([elapsed], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        elapsed = float(t.item())
    frames = args.steps * world
    value = frames / elapsed

    # end to end through the public API: pinned host scene in, image out
    e2e = None
    if not args.no_e2e:
        host = {k: torch.from_numpy(np.ascontiguousarray(scene_np[k])).pin_memory() for k in render.SCENE_KEYS}
        dscene = {k: torch.empty_like(scene[k]) for k in render.SCENE_KEYS}
        himg = torch.empty((H, W, 3), dtype=torch.float32).pin_memory()
        h2d = sum(v.numel() * 4 for v in host.values())
        d2h = himg.numel() * 4
        k2 = max(3, min(args.steps, 20))
        for i in range(2):
            for k in render.SCENE_KEYS:
                dscene[k].copy_(host[k], non_blocking=True)
            r.forward(dscene, cams[i % 8])
            himg.copy_(r.image, non_blocking=True)
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for i in range(k2):
            for k in render.SCENE_KEYS:
                dscene[k].copy_(host[k], non_blocking=True)
            r.forward(dscene, cams[(rank + i) % 8])
            himg.copy_(r.image, non_blocking=True)
        b.record(stream)
        torch.cuda.synchronize()
        t2 = a.elapsed_time(b) / 1e3
        if world > 1:
            t = torch.tensor([t2], device=dev)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            t2 = float(t.item())
        e2e = {"value": k2 * world / t2, "unit": "frames/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h}

    result = None
    if rank == 0:
        result = summarize(args, r, scene, cams, stage_ms, elapsed, value, frames, e2e, clk.summary(),
                           launches_per_frame * args.steps, passes, world)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()
    return result


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
    b_sort = sort_bytes(keys, passes)
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
    flops = evals * (11.0 + 8.0 * math.pi / 4.0)
    ms = stage_ms["rasterize"]
    sm_count = torch.cuda.get_device_properties(0).multi_processor_count
    peak_tflops = sm_count * 128 * 2 * peaks["sm_max_mhz"] * 1e6 / 1e12
    ach = flops / (ms * 1e-3) / 1e12
    stages["rasterize"] = {"ms": round(ms, 4), "bound": "alu", "alg_evals": int(evals),
                           "achieved_tflops": round(ach, 3), "peak_tflops": round(peak_tflops, 2),
                           "frac": round(ach / peak_tflops, 4)}
    dom = max(STAGES, key=lambda s: stage_ms[s])
    d = stages[dom]
    if d["bound"] == "hbm":
        roof = {"kernel": dom, "bound": "hbm", "achieved": d["achieved_gbs"], "peak": peaks["hbm_gbs"],
                "unit": "GB/s", "frac": d["frac"], "traffic": None, "peak_source": peaks["source"]}
    else:
        roof = {"kernel": dom, "bound": "alu", "achieved": d["achieved_tflops"], "peak": d["peak_tflops"],
                "unit": "TFLOP/s", "frac": d["frac"], "traffic": None,
                "peak_source": "derived: SMs x 128 FP32 lanes x 2 x max SM clock"}
    out = {
        "metric": METRIC, "value": round(value, 2), "unit": "frames/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(elapsed / args.steps * 1e3, 4),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic (seeded 64-cluster scene standing in for the paper's trained captures)",
        "config": {"workload": WORKLOADS[args.workload]["desc"], "tile": r.tile, "digit_bits": args.digit_bits,
                   "key_capacity": r.key_capacity, "mean_pairs_per_frame": int(keys),
                   "mean_visible": int(vis), "l2": "inputs larger than L2 (236 MB scene per frame)",
                   "parallelism": f"replicas x{world} (independent frames)"},
        "stages_ms": {s: round(stage_ms[s], 4) for s in STAGES},
        "stages": stages,
        "roofline": roof,
        "e2e": e2e,
        "gpu_launches": launches,
        "clocks": clocks,
    }
    if not args.no_cpu and world == 1:
        out["cpu_baseline"] = cpu_baseline(args)
    return out


def cpu_baseline(args, frames=2):
    """The FP64 oracle as it stands, single-threaded on the host, over whole
    frames of the same workload (bounded: `frames` frames)."""
    import oracle
    scene_np, cams = workload(args.workload)
    oracle.build()
    t = time.perf_counter()
    for k in range(frames):
        oracle.render(scene_np, cams[k])
    dt = time.perf_counter() - t
    return {"value": round(frames / dt, 4), "unit": "frames/s", "cores": 1, "kind": "oracle",
            "sample": f"{frames} full frames (poses 0..{frames - 1}) of the same workload, FP64 C oracle"}


# ------------------------------------------------------------- reference

def run_reference(args):
    """The FP64 oracle timed on the host cores; each step renders a 1/16
    sample of the scene's Gaussians (every 16th, same cameras) so the run
    stays within minutes; frames/s scales by that fraction."""
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return None
    import oracle
    oracle.build()
    scene_np, cams = workload(args.workload)
    frac = 16
    sub = {k: np.ascontiguousarray(v[::frac]) for k, v in scene_np.items()}
    for i in range(args.warmup):
        oracle.render(sub, cams[i % 8])
    t = time.perf_counter()
    for i in range(args.steps):
        oracle.render(sub, cams[i % 8])
    dt = time.perf_counter() - t
    value = args.steps / frac / dt
    return {"impl": "reference", "metric": METRIC, "value": round(value, 4), "unit": "frames/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(dt / args.steps * 1e3, 3), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOADS[args.workload]["desc"]},
            "cpu_baseline": {"value": round(value, 4), "unit": "frames/s", "cores": 1, "kind": "oracle",
                             "sample": f"each step: every {frac}th Gaussian of the scene, full image"},
            "e2e": {"value": round(value, 4), "unit": "frames/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="hd", choices=sorted(WORKLOADS))
    ap.add_argument("--tile", type=int, default=16)
    ap.add_argument("--digit-bits", type=int, default=8)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    res = run_reference(args) if args.impl == "reference" else run_ours(args)
    if res is not None:
        print(json.dumps(res), flush=True)


if __name__ == "__main__":
    main()
