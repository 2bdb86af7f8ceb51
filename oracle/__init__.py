"""FP64 CPU oracle for the 3DGS render path (test infrastructure).

Only the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline
leg import this package; the library never does. The arithmetic lives in
``ws_oracle.c`` (plain C, double precision); this module compiles it with gcc
on first use and marshals numpy arrays through ctypes. Function docstrings
name the paper passage each step follows; the C file states the readings
taken where the paper is silent.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ws_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "libws_oracle.so")
_lock = threading.Lock()
_lib = None

DEFAULTS = {"tile": 16, "dilation": 0.3, "guard": 1.3, "amb_px_rel": 1e-6, "amb_alpha": 1e-4, "flags": 0}
NO_OPACITY_CULL, NO_AABB_CULL, FIXED_RADIUS, PACKED = 1, 2, 8, 16
REASONS = {0: "visible", 1: "opacity", 2: "quat", 3: "near", 4: "det", 5: "offscreen"}


def build(force=False):
    """Compile ws_oracle.c into a shared library (gcc, -ffp-contract=off so the
    float32 depth is evaluated with every operation rounded)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC):
        return _LIB_PATH
    tmp = _LIB_PATH + f".{os.getpid()}.tmp"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
                           "-fno-fast-math", "-o", tmp, _SRC, "-lm"])
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Camera(C.Structure):
    _fields_ = [("viewmat", C.c_double * 12), ("fx", C.c_double), ("fy", C.c_double),
                ("cx", C.c_double), ("cy", C.c_double), ("width", C.c_int32),
                ("height", C.c_int32), ("znear", C.c_double), ("bg", C.c_double * 3)]


class _Config(C.Structure):
    _fields_ = [("tile", C.c_int32), ("dilation", C.c_double), ("guard", C.c_double),
                ("amb_px_rel", C.c_double), ("amb_alpha", C.c_double), ("flags", C.c_int32)]


_D = C.POINTER(C.c_double)
_F = C.POINTER(C.c_float)
_I32 = C.POINTER(C.c_int32)
_I64 = C.POINTER(C.c_int64)
_U8 = C.POINTER(C.c_uint8)
_U32 = C.POINTER(C.c_uint32)
_U64 = C.POINTER(C.c_uint64)


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(build())
            L.or_sh_basis.argtypes = [_D, _D]
            L.or_sh_basis_cart.argtypes = [_D, _D, _D]
            L.or_depth32.argtypes = [_D, _D]
            L.or_depth32.restype = C.c_float
            L.or_preprocess.argtypes = [C.c_int64, _D, _D, _D, _D, _D, C.POINTER(_Camera),
                                        C.POINTER(_Config), _D, _D, _D, _F, _D, _D, _D,
                                        _I32, _I32, _I32, _I32, _U8]
            L.or_preprocess.restype = C.c_int64
            L.or_emit_keys.argtypes = [C.c_int64, _I32, _F, C.c_int32, _U64, _U32, _I64]
            L.or_emit_keys.restype = C.c_int64
            L.or_sort_pairs.argtypes = [C.c_int64, _U64, _U32]
            L.or_tile_ranges.argtypes = [C.c_int64, _U64, C.c_int64, _I64]
            L.or_blend_tiles.argtypes = [C.POINTER(_Camera), C.POINTER(_Config), _D, _D, _D, _D,
                                         _U32, _I64, C.c_int64, _I64, _D, _D, _I64, C.POINTER(C.c_int32),
                                         _D, _D, _I64]
            L.or_blend_brute.argtypes = [C.POINTER(_Camera), C.c_int64, _D, _D, _D, _D, _F, _I32, _D, _D]
            L.or_loss_grad.argtypes = [C.c_int64, _D, _D, _D, _D, _D, C.POINTER(_Camera),
                                       C.POINTER(_Config), _D, _D, _D, _D, _D, _D, _D, _U64]
            L.or_loss_grad.restype = C.c_double
            L.or_round_f16.argtypes = [C.c_double]
            L.or_round_f16.restype = C.c_double
            L.or_axes.argtypes = [C.c_double, C.c_double, C.c_double, _D, _D]
            _lib = L
    return _lib


def _p(a, t):
    return a.ctypes.data_as(t)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def round_f16(x):
    """Nearest IEEE binary16 value of each double, ties to even (§3.2's
    packed axes)."""
    x = np.asarray(x, dtype=np.float64)
    return np.vectorize(lambda v: lib().or_round_f16(float(v)), otypes=[np.float64])(x)


def axes(sxx, sxy, syy):
    """Major and minor ellipse axes (v1, v2) of a 2D covariance, with
    v1 v1^T + v2 v2^T = [[sxx, sxy], [sxy, syy]] (§3.2's packed axes)."""
    v1 = np.zeros(2)
    v2 = np.zeros(2)
    lib().or_axes(float(sxx), float(sxy), float(syy), _p(v1, _D), _p(v2, _D))
    return v1, v2


def camera(cam):
    c = _Camera()
    vm = np.asarray(cam["viewmat"], dtype=np.float64).reshape(12)
    for i in range(12):
        c.viewmat[i] = vm[i]
    c.fx, c.fy, c.cx, c.cy = cam["fx"], cam["fy"], cam["cx"], cam["cy"]
    c.width, c.height = cam["width"], cam["height"]
    c.znear = cam["znear"]
    for i in range(3):
        c.bg[i] = cam["bg"][i]
    return c


def config(**kw):
    d = dict(DEFAULTS)
    d.update({k: v for k, v in kw.items() if v is not None})
    return _Config(int(d["tile"]), float(d["dilation"]), float(d["guard"]),
                   float(d["amb_px_rel"]), float(d["amb_alpha"]), int(d["flags"]))


def tiles(cam, tile=16):
    return (cam["width"] + tile - 1) // tile, (cam["height"] + tile - 1) // tile


# ------------------------------------------------------------------ SH

def sh_basis(d):
    """Real SH basis of degree 3 at unit direction d (§2.1), from the Legendre definition."""
    d = _f64(d)
    y = np.zeros(16)
    lib().or_sh_basis(_p(d, _D), _p(y, _D))
    return y


def sh_basis_cart(d):
    """Cartesian-polynomial form of the same basis and its gradient [16, 3]."""
    d = _f64(d)
    y = np.zeros(16)
    g = np.zeros((16, 3))
    lib().or_sh_basis_cart(_p(d, _D), _p(y, _D), _p(g, _D))
    return y, g


def depth32(x, viewmat):
    x = _f64(x)
    v = _f64(np.asarray(viewmat).reshape(12))
    return np.float32(lib().or_depth32(_p(x, _D), _p(v, _D)))


# ---------------------------------------------------------- pipeline steps

def preprocess(scene, cam, **cfg):
    """Per-Gaussian pre-processing (§3.2, §2.1, §3.4): projection, SH colour,
    culling, opacity-aware extent and tile rectangle."""
    n = scene["means"].shape[0]
    means, ls, qs = _f64(scene["means"]), _f64(scene["log_scales"]), _f64(scene["quats"])
    lg, sh = _f64(scene["opacity_logits"]), _f64(scene["sh"])
    out = {
        "mean2d": np.zeros((n, 2)), "cov2d": np.zeros((n, 3)), "conic": np.zeros((n, 3)),
        "depth": np.zeros(n, np.float32), "rgb": np.zeros((n, 3)), "opacity": np.zeros(n),
        "extent": np.zeros((n, 2)), "rect": np.zeros((n, 4), np.int32),
        "rect_exp": np.zeros((n, 4), np.int32), "touched": np.zeros(n, np.int32),
        "reason": np.zeros(n, np.int32), "amb": np.zeros(n, np.uint8),
    }
    c, g = camera(cam), config(**cfg)
    out["visible"] = lib().or_preprocess(
        n, _p(means, _D), _p(ls, _D), _p(qs, _D), _p(lg, _D), _p(sh, _D), C.byref(c), C.byref(g),
        _p(out["mean2d"], _D), _p(out["cov2d"], _D), _p(out["conic"], _D), _p(out["depth"], _F),
        _p(out["rgb"], _D), _p(out["opacity"], _D), _p(out["extent"], _D), _p(out["rect"], _I32),
        _p(out["rect_exp"], _I32), _p(out["touched"], _I32), _p(out["reason"], _I32),
        _p(out["amb"], _U8))
    return out


def emit_keys(rect, depth, tiles_x):
    """One (tile << 31 | depth bits, index) pair per overlapped tile, Gaussians
    in index order, tiles row-major (§3.4's <tile, splat> list)."""
    rect = np.ascontiguousarray(rect, dtype=np.int32)
    depth = np.ascontiguousarray(depth, dtype=np.float32)
    n = rect.shape[0]
    offsets = np.zeros(n + 1, np.int64)
    k = lib().or_emit_keys(n, _p(rect, _I32), _p(depth, _F), int(tiles_x), None, None, _p(offsets, _I64))
    keys = np.zeros(max(k, 1), np.uint64)
    vals = np.zeros(max(k, 1), np.uint32)
    lib().or_emit_keys(n, _p(rect, _I32), _p(depth, _F), int(tiles_x), _p(keys, _U64), _p(vals, _U32),
                       _p(offsets, _I64))
    return keys[:k], vals[:k], offsets


def sort_pairs(keys, vals):
    """Stable sort by key (§3.3.2); returns sorted copies."""
    k = np.array(keys, dtype=np.uint64, copy=True)
    v = np.array(vals, dtype=np.uint32, copy=True)
    lib().or_sort_pairs(k.size, _p(k, _U64), _p(v, _U32))
    return k, v


def tile_ranges(keys, ntiles):
    keys = np.ascontiguousarray(keys, dtype=np.uint64)
    r = np.zeros((ntiles, 2), np.int64)
    lib().or_tile_ranges(keys.size, _p(keys, _U64), int(ntiles), _p(r, _I64))
    return r


def blend_tiles(cam, proj, vals, ranges, tile_list=None, **cfg):
    """Front-to-back compositing (§2.1) over each tile's sorted list."""
    h, w = cam["height"], cam["width"]
    out = {"image": np.zeros((h, w, 3)), "t_final": np.ones((h, w)),
           "last_gid": np.full((h, w), -1, np.int64), "n_amb": np.zeros((h, w), np.int32),
           "alt_image": np.zeros((h, w, 3)), "alt_t_final": np.ones((h, w)),
           "alt_last_gid": np.full((h, w), -1, np.int64)}
    vals = np.ascontiguousarray(vals, dtype=np.uint32)
    ranges = np.ascontiguousarray(ranges, dtype=np.int64)
    tl = None if tile_list is None else np.ascontiguousarray(tile_list, dtype=np.int64)
    c, g = camera(cam), config(**cfg)
    lib().or_blend_tiles(C.byref(c), C.byref(g), _p(proj["mean2d"], _D), _p(proj["conic"], _D),
                         _p(proj["opacity"], _D), _p(proj["rgb"], _D),
                         _p(vals if vals.size else np.zeros(1, np.uint32), _U32), _p(ranges, _I64),
                         0 if tl is None else tl.size, None if tl is None else _p(tl, _I64),
                         _p(out["image"], _D), _p(out["t_final"], _D), _p(out["last_gid"], _I64),
                         out["n_amb"].ctypes.data_as(C.POINTER(C.c_int32)), _p(out["alt_image"], _D),
                         _p(out["alt_t_final"], _D), _p(out["alt_last_gid"], _I64))
    return out


def blend_brute(cam, proj):
    """Per pixel over all visible splats, back to front with "over" (§2.1)."""
    h, w = cam["height"], cam["width"]
    img = np.zeros((h, w, 3))
    tf = np.zeros((h, w))
    n = proj["mean2d"].shape[0]
    c = camera(cam)
    lib().or_blend_brute(C.byref(c), n, _p(proj["mean2d"], _D), _p(proj["conic"], _D),
                         _p(proj["opacity"], _D), _p(proj["rgb"], _D), _p(proj["depth"], _F),
                         _p(proj["touched"], _I32), _p(img, _D), _p(tf, _D))
    return img, tf


def render(scene, cam, tile_list=None, **cfg):
    """Whole forward path. The canonical key list (from the canonical rects)
    is returned for bit-exact comparison; the image is composited over lists
    built from the widened rects so that every pair the GPU may evaluate is
    decided (and flagged when ambiguous) by the oracle."""
    tile = cfg.get("tile") or DEFAULTS["tile"]
    tx, ty = tiles(cam, tile)
    proj = preprocess(scene, cam, **cfg)
    keys, vals, offsets = emit_keys(proj["rect"], proj["depth"], tx)
    skeys, svals = sort_pairs(keys, vals)
    ekeys, evals, _ = emit_keys(proj["rect_exp"], proj["depth"], tx)
    ekeys, evals = sort_pairs(ekeys, evals)
    eranges = tile_ranges(ekeys, tx * ty)
    out = blend_tiles(cam, proj, evals, eranges, tile_list=tile_list, **cfg)
    out.update(proj=proj, keys=keys, vals=vals, offsets=offsets, sorted_keys=skeys,
               sorted_vals=svals, ranges=tile_ranges(skeys, tx * ty))
    return out


def loss_grad(scene, cam, target, grads=True, image=False, **cfg):
    """L = 1/2 ||C - target||^2 and its analytic FP64 gradient; also the
    decision fingerprint used to screen finite differences."""
    n = scene["means"].shape[0]
    means, ls, qs = _f64(scene["means"]), _f64(scene["log_scales"]), _f64(scene["quats"])
    lg, sh = _f64(scene["opacity_logits"]), _f64(scene["sh"])
    tgt = _f64(target)
    c, g = camera(cam), config(**cfg)
    fp = C.c_uint64(0)
    img = np.zeros((cam["height"], cam["width"], 3)) if image else None
    if grads:
        out = {"means": np.zeros((n, 3)), "log_scales": np.zeros((n, 3)), "quats": np.zeros((n, 4)),
               "opacity_logits": np.zeros(n), "sh": np.zeros((n, 16, 3))}
        gp = [_p(out[k], _D) for k in ("means", "log_scales", "quats", "opacity_logits", "sh")]
    else:
        out, gp = None, [None] * 5
    loss = lib().or_loss_grad(n, _p(means, _D), _p(ls, _D), _p(qs, _D), _p(lg, _D), _p(sh, _D),
                              C.byref(c), C.byref(g), _p(tgt, _D),
                              None if img is None else _p(img, _D), *gp, C.byref(fp))
    return {"loss": loss, "grads": out, "fingerprint": fp.value, "image": img}
