"""Seeded synthetic scenes and cameras.

This module only draws inputs: it holds none of the render path's
arithmetic (no projection, colour, culling, sorting or blending), so both the
CUDA path and the FP64 oracle can be fed from it without sharing method code.

The paper evaluates on trained 3DGS scenes (bicycle, garden, truck, ... with
0.34M-6.1M splats, SH degree 3; §4.1 and Table 3) that are not available here.
These generators stand in for them at the same splat counts: Gaussian
clusters with anisotropic spreads, log-normal scales, a heavy tail of
near-transparent splats (to exercise opacity culling, §3.4) and degree-3 SH
coefficients, seen from cameras on an orbit.

All arrays are float32, C-contiguous, drawn with numpy's PCG64
(``np.random.default_rng(seed)``).

Layout of a scene (N Gaussians):
    means          [N, 3]      world position X
    log_scales     [N, 3]      log of the per-axis standard deviations
    quats          [N, 4]      rotation quaternion (w, x, y, z), unit norm
    opacity_logits [N]         logit of the peak opacity sigma
    sh             [N, 16, 3]  SH coefficients, degree 3, coefficient-major

A camera is a dict with ``viewmat`` (3x4 row-major world->camera [R|t],
OpenCV axes: x right, y down, z forward), ``fx, fy, cx, cy`` (pixels),
``width, height``, ``znear`` and ``bg`` (RGB background).
"""
from __future__ import annotations

import math

import numpy as np

SH_COEFFS = 16  # degree 3


def _random_unit_quats(rng, n):
    q = rng.standard_normal((n, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    return q


def _quat_to_matrix(q):
    """Rotation matrices of unit quaternions (w, x, y, z); used to draw cluster shapes."""
    w, x, y, z = q[:, 0], q[:, 1], q[:, 2], q[:, 3]
    r = np.empty((q.shape[0], 3, 3))
    r[:, 0, 0] = 1 - 2 * (y * y + z * z)
    r[:, 0, 1] = 2 * (x * y - w * z)
    r[:, 0, 2] = 2 * (x * z + w * y)
    r[:, 1, 0] = 2 * (x * y + w * z)
    r[:, 1, 1] = 1 - 2 * (x * x + z * z)
    r[:, 1, 2] = 2 * (y * z - w * x)
    r[:, 2, 0] = 2 * (x * z - w * y)
    r[:, 2, 1] = 2 * (y * z + w * x)
    r[:, 2, 2] = 1 - 2 * (x * x + y * y)
    return r


def _sh(rng, n, dc_std=0.5, rest_std=0.1):
    sh = np.empty((n, SH_COEFFS, 3), dtype=np.float64)
    sh[:, 0, :] = rng.normal(0.0, dc_std, (n, 3))
    sh[:, 1:, :] = rng.normal(0.0, rest_std, (n, SH_COEFFS - 1, 3))
    return sh


def _pack(means, log_scales, quats, logits, sh):
    return {
        "means": np.ascontiguousarray(means, dtype=np.float32),
        "log_scales": np.ascontiguousarray(log_scales, dtype=np.float32),
        "quats": np.ascontiguousarray(quats, dtype=np.float32),
        "opacity_logits": np.ascontiguousarray(logits, dtype=np.float32),
        "sh": np.ascontiguousarray(sh, dtype=np.float32),
    }


def uniform_scene(n, seed, extent=1.0, log_scale_mean=-4.0, log_scale_std=0.5,
                  logit_std=1.5):
    """Uniform cube scene: means U[-extent, extent]^3, log-scales N(mu, s),
    random unit quaternions, logits N(0, logit_std), SH DC N(0, .5), rest N(0, .1)."""
    rng = np.random.default_rng(seed)
    means = rng.uniform(-extent, extent, (n, 3))
    log_scales = rng.normal(log_scale_mean, log_scale_std, (n, 3))
    quats = _random_unit_quats(rng, n)
    logits = rng.normal(0.0, logit_std, n)
    sh = _sh(rng, n)
    return _pack(means, log_scales, quats, logits, sh)


def cluster_scene(n, seed, box=20.0, n_clusters=64, std_range=(0.3, 2.0),
                  log_scale_mean=-5.0, log_scale_std=0.8, low_opacity_frac=0.4):
    """Clustered scene standing in for a trained capture.

    ``n_clusters`` centres uniform in a cube of side ``box``; each cluster has a
    random orientation and per-axis spreads U(std_range) (scaled with the box);
    points are assigned uniformly to clusters. ``low_opacity_frac`` of the
    splats get sigma ~ LogUniform(1e-4, 0.05) (about 59% of these fall below
    1/255 and are culled); the rest get logit ~ N(0, 1.5) conditioned on
    sigma >= 0.05.
    """
    rng = np.random.default_rng(seed)
    half = box / 2.0
    scale = box / 20.0
    centres = rng.uniform(-half, half, (n_clusters, 3))
    crot = _quat_to_matrix(_random_unit_quats(rng, n_clusters))
    cstd = rng.uniform(std_range[0] * scale, std_range[1] * scale, (n_clusters, 3))
    assign = rng.integers(0, n_clusters, n)
    local = rng.standard_normal((n, 3)) * cstd[assign]
    means = centres[assign] + np.einsum("nij,nj->ni", crot[assign], local)
    log_scales = rng.normal(log_scale_mean, log_scale_std, (n, 3)) + math.log(scale)
    quats = _random_unit_quats(rng, n)
    logits = np.empty(n)
    low = rng.random(n) < low_opacity_frac
    n_low = int(low.sum())
    sig = np.exp(rng.uniform(math.log(1e-4), math.log(0.05), n_low))
    logits[low] = np.log(sig) - np.log1p(-sig)
    lo_logit = math.log(0.05) - math.log(0.95)
    hi = np.flatnonzero(~low)
    vals = rng.normal(0.0, 1.5, hi.size)
    bad = vals < lo_logit
    while bad.any():
        vals[bad] = rng.normal(0.0, 1.5, int(bad.sum()))
        bad = vals < lo_logit
    logits[hi] = vals
    sh = _sh(rng, n)
    return _pack(means, log_scales, quats, logits, sh)


def look_at_camera(position, target, width, height, fov_x_deg=60.0, up=(0.0, 0.0, 1.0),
                   znear=0.2, bg=(0.0, 0.0, 0.0), f=None):
    """Pinhole camera at ``position`` looking at ``target`` (OpenCV axes)."""
    c = np.asarray(position, dtype=np.float64)
    fwd = np.asarray(target, dtype=np.float64) - c
    fwd /= np.linalg.norm(fwd)
    right = np.cross(fwd, np.asarray(up, dtype=np.float64))
    right /= np.linalg.norm(right)
    down = np.cross(fwd, right)
    rot = np.stack([right, down, fwd])
    t = -rot @ c
    if f is None:
        f = width / (2.0 * math.tan(math.radians(fov_x_deg) / 2.0))
    viewmat = np.concatenate([rot, t[:, None]], axis=1).astype(np.float32)
    return {
        "viewmat": viewmat, "fx": float(np.float32(f)), "fy": float(np.float32(f)),
        "cx": width / 2.0, "cy": height / 2.0, "width": int(width), "height": int(height),
        "znear": float(np.float32(znear)), "bg": tuple(float(np.float32(b)) for b in bg),
    }


def orbit_pose(k, seed, radius, height, n_poses=8):
    """k-th of ``n_poses`` camera positions on a horizontal orbit with a seeded azimuth jitter."""
    rng = np.random.default_rng(seed)
    az = 2.0 * math.pi * k / n_poses + rng.uniform(-0.1, 0.1)
    return (radius * math.cos(az), radius * math.sin(az), height)


# ---------------------------------------------------------------- workloads

def small_forward():
    """10,000 Gaussians in [-1,1]^3, 256x256, camera at distance 3, fx = fy = 256."""
    scene = uniform_scene(10_000, seed=0)
    cam = {
        "viewmat": np.array([[1, 0, 0, 0], [0, 1, 0, 0], [0, 0, 1, 3]], dtype=np.float32),
        "fx": 256.0, "fy": 256.0, "cx": 128.0, "cy": 128.0, "width": 256, "height": 256,
        "znear": float(np.float32(0.2)), "bg": (0.0, 0.0, 0.0),
    }
    return scene, cam


def hd_scene(n=1_000_000, seed=1):
    """1M-Gaussian clustered scene in a 20-unit box (the 1080p workload)."""
    return cluster_scene(n, seed=seed, box=20.0)


def hd_camera(k, width=1920, height=1080):
    """Pose k (0..7) on the orbit of radius 25 at height 5, 60 degree horizontal FOV."""
    pos = orbit_pose(k, seed=100 + k, radius=25.0, height=5.0)
    return look_at_camera(pos, (0.0, 0.0, 0.0), width, height)


def uhd_scene(n=6_000_000, seed=3):
    """6M-Gaussian clustered scene in a 60-unit box (the 4K workload)."""
    return cluster_scene(n, seed=seed, box=60.0)


def uhd_camera(k, width=3840, height=2160):
    pos = orbit_pose(k, seed=100 + k, radius=75.0, height=15.0)
    return look_at_camera(pos, (0.0, 0.0, 0.0), width, height)


def sort_keys(n=4_194_304, seed=2, tiles=8160):
    """Standalone (tile, depth) key array: tile U{0..tiles-1}, depth U(1, 60) as float32 bits.

    The key packs the tile id above the 31 low bits that hold the positive
    float32 depth's bit pattern (its sign bit is always 0)."""
    rng = np.random.default_rng(seed)
    tile = rng.integers(0, tiles, n).astype(np.uint64)
    depth = rng.uniform(1.0, 60.0, n).astype(np.float32).view(np.uint32).astype(np.uint64)
    keys = (tile << np.uint64(31)) | depth
    vals = np.arange(n, dtype=np.uint32)
    return keys, vals


def grad_scene():
    """500k-Gaussian clustered scene, 1280x720 camera and a U[0,1) target image."""
    scene = cluster_scene(500_000, seed=4, box=20.0)
    cam = hd_camera(0, width=1280, height=720)
    target = np.random.default_rng(5).random((720, 1280, 3)).astype(np.float32)
    return scene, cam, target


def gradcheck_scene():
    """64 Gaussians (uniform generator), 32x32 image, f = 32, camera at distance 3."""
    scene = uniform_scene(64, seed=6)
    cam = {
        "viewmat": np.array([[1, 0, 0, 0], [0, 1, 0, 0], [0, 0, 1, 3]], dtype=np.float32),
        "fx": 32.0, "fy": 32.0, "cx": 16.0, "cy": 16.0, "width": 32, "height": 32,
        "znear": float(np.float32(0.2)), "bg": (0.0, 0.0, 0.0),
    }
    target = np.random.default_rng(60).random((32, 32, 3)).astype(np.float32)
    return scene, cam, target


def batch_views(n_views=64, seed0=200):
    """Cameras of uneven resolution (W ~ U{320..1920}, H ~ U{240..1080}) on the hd orbit."""
    cams = []
    for v in range(n_views):
        rng = np.random.default_rng(seed0 + v)
        w = int(rng.integers(320, 1921))
        h = int(rng.integers(240, 1081))
        az = rng.uniform(0.0, 2.0 * math.pi)
        pos = (25.0 * math.cos(az), 25.0 * math.sin(az), 5.0)
        cams.append(look_at_camera(pos, (0.0, 0.0, 0.0), w, h))
    return cams


def batch_scene(n=2_000_000, seed=7):
    return cluster_scene(n, seed=seed, box=20.0)
