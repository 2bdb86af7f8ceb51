"""Autotuner for the batched path: tile size x sort digit width.

For one workload (scene size, the batch's resolutions, GPU) it builds a
BatchRenderer per candidate, captures one training step (forward + residual
+ backward) as a CUDA graph, times a few replays with CUDA events and keeps
the fastest. Results are cached as JSON keyed by a workload signature, so a
second run of the same workload skips the search. Every candidate produces
the same images and gradients; only the speed differs.
"""
from __future__ import annotations

import hashlib
import json
import math
import os

import torch

from .batch import BatchRenderer

TILES = (8, 16, 32)
DIGITS = (8, 10, 11)


def cache_path():
    base = os.environ.get("XDG_CACHE_HOME") or os.path.join(os.path.expanduser("~"), ".cache")
    return os.path.join(base, "websplat", "autotune.json")


def signature(n, cams, device=None):
    res = ",".join(f"{c['width']}x{c['height']}" for c in cams)
    name = torch.cuda.get_device_name(device)
    h = hashlib.sha1(res.encode()).hexdigest()[:16]
    return f"{name}|n={n}|views={len(cams)}|res={h}"


def _load():
    try:
        with open(cache_path()) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _save(db):
    p = cache_path()
    try:
        os.makedirs(os.path.dirname(p), exist_ok=True)
        tmp = p + f".{os.getpid()}.tmp"
        with open(tmp, "w") as f:
            json.dump(db, f, indent=1, sort_keys=True)
        os.replace(tmp, p)
    except OSError:
        pass  # a read-only home only loses the cache


def measure_capacity(scene, cams, tile, digit_bits):
    """Pairs one forward of the batch produces (probe with generous capacity)."""
    n = scene["means"].shape[0]
    probe = BatchRenderer(n, cams, tile=tile, digit_bits=digit_bits,
                          key_capacity=min((1 << 31) - 1, 3 * n * len(cams)))
    probe.forward(scene)
    probe.check_status()
    k = probe.key_count()
    del probe
    torch.cuda.empty_cache()
    return k


def time_step(b, scene, target, reps=3):
    g = b.capture(scene, target)
    g.replay()
    torch.cuda.synchronize()
    start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    start.record()
    for _ in range(reps):
        g.replay()
    end.record()
    torch.cuda.synchronize()
    ms = start.elapsed_time(end) / reps
    del g
    return ms


def tune(scene, cams, target, tiles=TILES, digits=DIGITS, reps=3, use_cache=True, log=None):
    """Returns {"tile", "digit_bits", "key_capacity", "ms", "table"} for the workload."""
    n = scene["means"].shape[0]
    sig = signature(n, cams)
    db = _load() if use_cache else {}
    if use_cache and sig in db:
        return dict(db[sig], cached=True)
    table = []
    best = None
    for tile in tiles:
        k = measure_capacity(scene, cams, tile, digits[0])
        cap = min((1 << 31) - 1, int(math.ceil(k * 1.1 / 4096) * 4096) + 4096)
        for bits in digits:
            b = BatchRenderer(n, cams, tile=tile, digit_bits=bits, key_capacity=cap)
            ms = time_step(b, scene, target, reps)
            b.check_status()
            del b
            torch.cuda.empty_cache()
            table.append({"tile": tile, "digit_bits": bits, "ms": round(ms, 4), "key_capacity": cap})
            if log:
                log(f"autotune tile={tile} digit_bits={bits}: {ms:.3f} ms/step")
            if best is None or ms < best["ms"]:
                best = {"tile": tile, "digit_bits": bits, "key_capacity": cap, "ms": round(ms, 4)}
    best["table"] = table
    if use_cache:
        db[sig] = best
        _save(db)
    return dict(best, cached=False)
