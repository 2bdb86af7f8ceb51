"""Thin Python binding of the C ABI in include/websplat.h.

Argument marshalling only: every function here has the name of the C entry
point it forwards to, takes torch tensors (device memory) and plain values,
passes their data pointers and the current CUDA stream through ctypes, and
turns a non-zero status into an exception. All arithmetic runs in the CUDA
kernels of libwebsplat.so. There is no fallback: if the library is missing
the first call raises.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import torch

from . import build as _build

_lock = threading.Lock()
_lib = None

WS_OK, WS_ERR_INVALID_ARG, WS_ERR_CUDA, WS_ERR_CAPACITY, WS_ERR_TIMEOUT, WS_ERR_UNSUPPORTED = range(6)
WS_FLAG_CAPACITY, WS_FLAG_TIMEOUT = 1, 2
WS_CFG_NO_OPACITY_CULL, WS_CFG_NO_AABB_CULL, WS_CFG_SORT_LOOKBACK, WS_CFG_FIXED_RADIUS = 1, 2, 4, 8
WS_CFG_SORT_SEGMENTED = 16
WS_CFG_PERSISTENT = 32
WS_CFG_RANGES_GIVEN = 64
WS_CFG_BOX_MASKS = 128
WS_ABI_VERSION = 2
WS_SPLAT_FLOATS = 12  # floats per splat record: centre hi/lo (4), conic (3), sigma, colour (3), axis word

EXPORTS = ("ws_abi_version", "ws_status_string", "ws_workspace_bytes", "ws_preprocess", "ws_cull",
           "ws_sort", "ws_sort_noalloc", "ws_sort_noalloc_max_keys", "ws_rasterize",
           "ws_rasterize_backward", "ws_read_status", "ws_batch_max_views", "ws_batch_workspace_bytes",
           "ws_preprocess_batch", "ws_cull_batch", "ws_rasterize_batch", "ws_rasterize_backward_batch",
           "ws_image_residual", "ws_sort_test_stalled_tile", "ws_render_train_l2", "ws_render_train_l2_batch",
           "ws_sort_tiles", "ws_render_frame_host", "ws_cull_sort_tiles")


class WsError(RuntimeError):
    def __init__(self, call, status):
        msg = lib().ws_status_string(status).decode()
        super().__init__(f"{call} failed: {msg} (status {status})")
        self.status = status


class Camera(C.Structure):
    _fields_ = [("viewmat", C.c_float * 12), ("fx", C.c_float), ("fy", C.c_float), ("cx", C.c_float),
                ("cy", C.c_float), ("width", C.c_int32), ("height", C.c_int32), ("znear", C.c_float),
                ("bg", C.c_float * 3)]


class FrameBuffers(C.Structure):
    _fields_ = [(name, C.c_void_p) for name in (
        "means", "log_scales", "quats", "opacity_logits", "sh", "splats", "depth", "rect", "tiles_touched",
        "offsets", "keys", "keys_alt", "vals", "vals_alt", "num_keys", "ranges", "image", "t_final",
        "n_contrib", "workspace")] + [("key_capacity", C.c_int64)]


class Config(C.Structure):
    _fields_ = [("tile", C.c_int32), ("digit_bits", C.c_int32), ("dilation", C.c_float),
                ("guard", C.c_float), ("flags", C.c_uint32)]


def camera(cam: dict) -> Camera:
    c = Camera()
    vm = [float(v) for row in cam["viewmat"] for v in row] if hasattr(cam["viewmat"][0], "__len__") \
        else [float(v) for v in cam["viewmat"]]
    for i in range(12):
        c.viewmat[i] = vm[i]
    c.fx, c.fy, c.cx, c.cy = cam["fx"], cam["fy"], cam["cx"], cam["cy"]
    c.width, c.height, c.znear = int(cam["width"]), int(cam["height"]), cam["znear"]
    for i in range(3):
        c.bg[i] = cam["bg"][i]
    return c


def config(tile=16, digit_bits=8, dilation=0.3, guard=1.3, flags=0) -> Config:
    return Config(int(tile), int(digit_bits), float(dilation), float(guard), int(flags))


def lib():
    """The loaded libwebsplat.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.LIB_PATH
            if not os.path.exists(path):
                raise RuntimeError(f"{path} is missing: build it with "
                                   "`python -m paper_2602_03207_gb300.build` (needs nvcc)")
            L = C.CDLL(path)
            P, I64, I32, U32 = C.c_void_p, C.c_int64, C.c_int32, C.c_uint32
            cam_p, cfg_p = C.POINTER(Camera), C.POINTER(Config)
            L.ws_abi_version.restype = I32
            L.ws_status_string.argtypes = [I32]
            L.ws_status_string.restype = C.c_char_p
            L.ws_workspace_bytes.argtypes = [I64, I64, cam_p, cfg_p]
            L.ws_workspace_bytes.restype = C.c_size_t
            L.ws_preprocess.argtypes = [I64, P, P, P, P, P, cam_p, cfg_p, P, P, P, P, P]
            L.ws_cull.argtypes = [I64, P, P, P, cam_p, cfg_p, P, P, P, I64, P, P, P]
            L.ws_sort.argtypes = [P, I64, I32, I32, P, P, P, P, cfg_p, P, C.POINTER(I32), P]
            L.ws_rasterize.argtypes = [P, P, P, P, cam_p, cfg_p, P, P, P, P, P]
            L.ws_preprocess_packed.argtypes = [I64, P, P, P, P, P, cam_p, cfg_p, P, P, P, P, P, P, P]
            L.ws_quads_workspace_bytes.argtypes = [I64, I64, cam_p, cfg_p]
            L.ws_quads_workspace_bytes.restype = C.c_size_t
            L.ws_render_quads.argtypes = [I64, P, P, P, cam_p, cfg_p, I64, P, P, P, P, P, P, P, P, P]
            L.ws_rasterize_packed.argtypes = [P, P, P, P, P, P, cam_p, cfg_p, P, P, P, P, P]
            L.ws_rasterize_backward.argtypes = [I64, P, P, P, P, P, cam_p, cfg_p, P, P, P, P, P, P, P, P,
                                                P, I64, P, P, P, P, P, P, P]
            L.ws_sort_test_stalled_tile.argtypes = [P, I64, I32, I32, P, P, P, P, cfg_p, P, I32, C.POINTER(I32), P]
            L.ws_sort_test_stalled_tile.restype = I32
            L.ws_sort_tiles.argtypes = [P, I64, I32, P, P, P, P, cfg_p, P, P, I64, C.POINTER(I32), P]
            L.ws_sort_tiles.restype = I32
            L.ws_cull_sort_tiles.argtypes = [I64, P, P, P, cam_p, cfg_p, P, P, P, P, P, I64, P, P, P,
                                             C.POINTER(I32), P]
            L.ws_cull_sort_tiles.restype = I32
            L.ws_render_frame_host.argtypes = [I64, P, P, P, P, P, cam_p, cfg_p, C.POINTER(FrameBuffers), P, P]
            L.ws_render_frame_host.restype = I32
            L.ws_sort_noalloc.argtypes = [P, I64, I32, I32, P, P, P, P, I32, C.POINTER(I32), P]
            L.ws_sort_noalloc.restype = I32
            L.ws_sort_noalloc_max_keys.restype = I64
            L.ws_read_status.argtypes = [P, C.POINTER(U32), I32, P]
            L.ws_batch_max_views.restype = I32
            L.ws_batch_workspace_bytes.argtypes = [I64, I32, cam_p, I64, cfg_p]
            L.ws_batch_workspace_bytes.restype = C.c_size_t
            L.ws_preprocess_batch.argtypes = [I64, P, P, P, P, P, I32, cam_p, cfg_p, P, P, P, P, P]
            L.ws_cull_batch.argtypes = [I64, I32, cam_p, cfg_p, P, P, P, P, P, P, I64, P, P, P]
            L.ws_rasterize_batch.argtypes = [P, P, P, I64, P, I32, cam_p, cfg_p, P, P, P, P, P]
            L.ws_rasterize_backward_batch.argtypes = [I64, P, P, P, P, I32, cam_p, cfg_p, P, P, P, P, P,
                                                      P, P, P, P, I64, P, P, P, P, P, P, P]
            L.ws_image_residual.argtypes = [I64, P, P, P, P]
            L.ws_render_train_l2.argtypes = [I64, P, P, P, P, cam_p, cfg_p, P, P, P, P, P, P, P, P, I64, P, P, P, P,
                                             P, P, P, P, P, P, P]
            L.ws_render_train_l2_batch.argtypes = [I64, P, P, P, P, I32, cam_p, cfg_p, P, P, P, P, P, P, P, P, I64,
                                                   P, P, P, P, P, P, P, P, P, P, P]
            for name in ("ws_preprocess_batch", "ws_cull_batch", "ws_rasterize_batch", "ws_rasterize_backward_batch",
                         "ws_image_residual", "ws_sort_test_stalled_tile", "ws_render_train_l2",
                         "ws_render_train_l2_batch"):
                getattr(L, name).restype = I32
            for name in ("ws_preprocess", "ws_cull", "ws_sort", "ws_rasterize", "ws_rasterize_backward",
                         "ws_read_status"):
                getattr(L, name).restype = I32
            _lib = L
    return _lib


def _ptr(t):
    if t is None:
        return None
    if isinstance(t, torch.Tensor):
        if t.numel() and not t.is_cuda:
            raise ValueError("device tensor expected")
        return t.data_ptr() if t.numel() else None
    return int(t)


def _stream(stream):
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def _check(call, status):
    if status != WS_OK:
        raise WsError(call, status)


def ws_workspace_bytes(n, key_capacity, cam: Camera, cfg: Config) -> int:
    return int(lib().ws_workspace_bytes(int(n), int(key_capacity), C.byref(cam), C.byref(cfg)))


def ws_preprocess(n, means, log_scales, quats, opacity_logits, sh, cam, cfg, splats, depth, rect, tiles_touched,
                  stream=None):
    _check("ws_preprocess", lib().ws_preprocess(
        int(n), _ptr(means), _ptr(log_scales), _ptr(quats), _ptr(opacity_logits), _ptr(sh),
        C.byref(cam), C.byref(cfg), _ptr(splats), _ptr(depth), _ptr(rect), _ptr(tiles_touched), _stream(stream)))


def ws_cull(n, tiles_touched, rect, depth, cam, cfg, offsets, keys, vals, key_capacity, num_keys,
            workspace, stream=None):
    _check("ws_cull", lib().ws_cull(
        int(n), _ptr(tiles_touched), _ptr(rect), _ptr(depth), C.byref(cam), C.byref(cfg),
        _ptr(offsets), _ptr(keys), _ptr(vals), int(key_capacity), _ptr(num_keys), _ptr(workspace),
        _stream(stream)))


def ws_sort(num_keys, key_capacity, begin_bit, end_bit, keys, vals, keys_alt, vals_alt, cfg,
            workspace, stream=None) -> bool:
    """Returns True when the sorted data ended in the _alt buffers."""
    in_alt = C.c_int32(0)
    _check("ws_sort", lib().ws_sort(
        _ptr(num_keys), int(key_capacity), int(begin_bit), int(end_bit), _ptr(keys), _ptr(vals),
        _ptr(keys_alt), _ptr(vals_alt), C.byref(cfg), _ptr(workspace), C.byref(in_alt),
        _stream(stream)))
    return bool(in_alt.value)


def ws_sort_tiles(num_keys, key_capacity, end_bit, keys, vals, keys_alt, vals_alt, cfg, workspace, ranges, ntiles,
                  stream=None) -> bool:
    """Segmented sort that also writes the tile ranges; True when the result is in the _alt buffers."""
    in_alt = C.c_int32(0)
    _check("ws_sort_tiles", lib().ws_sort_tiles(
        _ptr(num_keys), int(key_capacity), int(end_bit), _ptr(keys), _ptr(vals), _ptr(keys_alt), _ptr(vals_alt),
        C.byref(cfg), _ptr(workspace), _ptr(ranges), int(ntiles), C.byref(in_alt), _stream(stream)))
    return bool(in_alt.value)


def ws_cull_sort_tiles(n, tiles_touched, rect, depth, cam, cfg, offsets, keys, vals, keys_alt, vals_alt,
                       key_capacity, num_keys, ranges, workspace, stream=None) -> bool:
    """ws_cull and ws_sort_tiles with the compaction fused into the sort's
    first partition pass; True when the sorted pairs are in the _alt buffers."""
    in_alt = C.c_int32(0)
    _check("ws_cull_sort_tiles", lib().ws_cull_sort_tiles(
        int(n), _ptr(tiles_touched), _ptr(rect), _ptr(depth), C.byref(cam), C.byref(cfg), _ptr(offsets),
        _ptr(keys), _ptr(vals), _ptr(keys_alt), _ptr(vals_alt), int(key_capacity), _ptr(num_keys), _ptr(ranges),
        _ptr(workspace), C.byref(in_alt), _stream(stream)))
    return bool(in_alt.value)


def ws_sort_test_stalled_tile(num_keys, key_capacity, begin_bit, end_bit, keys, vals, keys_alt, vals_alt, cfg,
                              workspace, stalled_tile, stream=None) -> bool:
    in_alt = C.c_int32(0)
    _check("ws_sort_test_stalled_tile", lib().ws_sort_test_stalled_tile(
        _ptr(num_keys), int(key_capacity), int(begin_bit), int(end_bit), _ptr(keys), _ptr(vals), _ptr(keys_alt),
        _ptr(vals_alt), C.byref(cfg), _ptr(workspace), int(stalled_tile), C.byref(in_alt), _stream(stream)))
    return bool(in_alt.value)


def ws_sort_noalloc_max_keys() -> int:
    return int(lib().ws_sort_noalloc_max_keys())


def ws_sort_noalloc(num_keys, key_capacity, begin_bit, end_bit, keys, vals, keys_alt, vals_alt, digit_bits=8,
                    stream=None) -> bool:
    """Workspace-free ws_sort (library-held scratch); True when the result is in the _alt buffers."""
    in_alt = C.c_int32(0)
    _check("ws_sort_noalloc", lib().ws_sort_noalloc(
        _ptr(num_keys), int(key_capacity), int(begin_bit), int(end_bit), _ptr(keys), _ptr(vals),
        _ptr(keys_alt), _ptr(vals_alt), int(digit_bits), C.byref(in_alt), _stream(stream)))
    return bool(in_alt.value)


def ws_rasterize(num_keys, keys, vals, splats, cam, cfg, ranges, image, t_final, n_contrib, stream=None):
    _check("ws_rasterize", lib().ws_rasterize(
        _ptr(num_keys), _ptr(keys), _ptr(vals), _ptr(splats), C.byref(cam), C.byref(cfg), _ptr(ranges), _ptr(image), _ptr(t_final), _ptr(n_contrib),
        _stream(stream)))


def ws_preprocess_packed(n, means, log_scales, quats, opacity_logits, sh, cam, cfg, mean2d, axes, rgba, depth,
                         rect, tiles_touched, stream=None):
    _check("ws_preprocess_packed", lib().ws_preprocess_packed(
        int(n), _ptr(means), _ptr(log_scales), _ptr(quats), _ptr(opacity_logits), _ptr(sh), C.byref(cam),
        C.byref(cfg), _ptr(mean2d), _ptr(axes), _ptr(rgba), _ptr(depth), _ptr(rect), _ptr(tiles_touched),
        _stream(stream)))


def ws_rasterize_packed(num_keys, keys, vals, mean2d, axes, rgba, cam, cfg, ranges, image, t_final, n_contrib,
                        stream=None):
    _check("ws_rasterize_packed", lib().ws_rasterize_packed(
        _ptr(num_keys), _ptr(keys), _ptr(vals), _ptr(mean2d), _ptr(axes), _ptr(rgba), C.byref(cam),
        C.byref(cfg), _ptr(ranges), _ptr(image), _ptr(t_final), _ptr(n_contrib), _stream(stream)))


def ws_quads_workspace_bytes(n, key_capacity, cam, cfg):
    return int(lib().ws_quads_workspace_bytes(int(n), int(key_capacity), C.byref(cam), C.byref(cfg)))


def ws_render_quads(n, splats, depth, tiles_touched, cam, cfg, key_capacity, keys, vals, keys_alt, vals_alt,
                    num_keys, image, t_final, workspace, stream=None):
    _check("ws_render_quads", lib().ws_render_quads(
        int(n), _ptr(splats), _ptr(depth), _ptr(tiles_touched),
        C.byref(cam), C.byref(cfg), int(key_capacity), _ptr(keys), _ptr(vals), _ptr(keys_alt), _ptr(vals_alt),
        _ptr(num_keys), _ptr(image), _ptr(t_final), _ptr(workspace), _stream(stream)))


def ws_rasterize_backward(n, means, log_scales, quats, opacity_logits, sh, cam, cfg, splats, rect, offsets,
                          tiles_touched, vals, ranges, t_final, n_contrib, d_image, key_capacity, d_means,
                          d_log_scales, d_quats, d_opacity_logits, d_sh, workspace, stream=None):
    _check("ws_rasterize_backward", lib().ws_rasterize_backward(
        int(n), _ptr(means), _ptr(log_scales), _ptr(quats), _ptr(opacity_logits), _ptr(sh), C.byref(cam),
        C.byref(cfg), _ptr(splats), _ptr(rect), _ptr(offsets),
        _ptr(tiles_touched), _ptr(vals), _ptr(ranges), _ptr(t_final), _ptr(n_contrib), _ptr(d_image),
        int(key_capacity), _ptr(d_means), _ptr(d_log_scales), _ptr(d_quats), _ptr(d_opacity_logits),
        _ptr(d_sh), _ptr(workspace), _stream(stream)))


def ws_read_status(workspace, clear=False, stream=None) -> int:
    flags = C.c_uint32(0)
    _check("ws_read_status", lib().ws_read_status(_ptr(workspace), C.byref(flags), int(bool(clear)),
                                                  _stream(stream)))
    return int(flags.value)


# ------------------------------------------------------------ batched views

def camera_array(cams):
    """ctypes array of ws_camera from a list of camera dicts."""
    arr = (Camera * len(cams))()
    for i, c in enumerate(cams):
        arr[i] = camera(c)
    return arr


def ws_batch_max_views() -> int:
    return int(lib().ws_batch_max_views())


def ws_batch_workspace_bytes(n, cams_arr, key_capacity, cfg) -> int:
    return int(lib().ws_batch_workspace_bytes(int(n), len(cams_arr), cams_arr, int(key_capacity), C.byref(cfg)))


def ws_preprocess_batch(n, means, log_scales, quats, opacity_logits, sh, cams_arr, cfg, splats, depth, rect,
                        tiles_touched, stream=None):
    _check("ws_preprocess_batch", lib().ws_preprocess_batch(
        int(n), _ptr(means), _ptr(log_scales), _ptr(quats), _ptr(opacity_logits), _ptr(sh), len(cams_arr),
        cams_arr, C.byref(cfg), _ptr(splats), _ptr(depth), _ptr(rect), _ptr(tiles_touched), _stream(stream)))


def ws_cull_batch(n, cams_arr, cfg, tiles_touched, rect, depth, offsets, keys, vals, key_capacity, num_keys,
                  workspace, stream=None):
    _check("ws_cull_batch", lib().ws_cull_batch(
        int(n), len(cams_arr), cams_arr, C.byref(cfg), _ptr(tiles_touched), _ptr(rect), _ptr(depth), _ptr(offsets),
        _ptr(keys), _ptr(vals), int(key_capacity), _ptr(num_keys), _ptr(workspace), _stream(stream)))


def ws_rasterize_batch(num_keys, keys, vals, n, splats, cams_arr, cfg, ranges, image, t_final, n_contrib,
                       stream=None):
    _check("ws_rasterize_batch", lib().ws_rasterize_batch(
        _ptr(num_keys), _ptr(keys), _ptr(vals), int(n), _ptr(splats), len(cams_arr), cams_arr, C.byref(cfg), _ptr(ranges), _ptr(image), _ptr(t_final), _ptr(n_contrib),
        _stream(stream)))


def ws_rasterize_backward_batch(n, means, log_scales, quats, sh, cams_arr, cfg, splats, rect, offsets,
                                tiles_touched, vals, ranges, t_final, n_contrib, d_image, key_capacity, d_means,
                                d_log_scales, d_quats, d_opacity_logits, d_sh, workspace, stream=None):
    _check("ws_rasterize_backward_batch", lib().ws_rasterize_backward_batch(
        int(n), _ptr(means), _ptr(log_scales), _ptr(quats), _ptr(sh), len(cams_arr), cams_arr, C.byref(cfg),
        _ptr(splats), _ptr(rect), _ptr(offsets), _ptr(tiles_touched),
        _ptr(vals), _ptr(ranges), _ptr(t_final), _ptr(n_contrib), _ptr(d_image), int(key_capacity), _ptr(d_means),
        _ptr(d_log_scales), _ptr(d_quats), _ptr(d_opacity_logits), _ptr(d_sh), _ptr(workspace), _stream(stream)))


def ws_image_residual(count, image, target, d_image, stream=None):
    _check("ws_image_residual", lib().ws_image_residual(int(count), _ptr(image), _ptr(target), _ptr(d_image),
                                                        _stream(stream)))


def ws_render_train_l2(n, means, log_scales, quats, sh, cam, cfg, num_keys, keys, vals, splats, rect, offsets,
                       tiles_touched, target, key_capacity, ranges, image, t_final, n_contrib, d_means, d_log_scales,
                       d_quats, d_opacity_logits, d_sh, workspace, stream=None):
    _check("ws_render_train_l2", lib().ws_render_train_l2(
        int(n), _ptr(means), _ptr(log_scales), _ptr(quats), _ptr(sh), C.byref(cam), C.byref(cfg), _ptr(num_keys),
        _ptr(keys), _ptr(vals), _ptr(splats), _ptr(rect), _ptr(offsets), _ptr(tiles_touched), _ptr(target),
        int(key_capacity), _ptr(ranges), _ptr(image), _ptr(t_final), _ptr(n_contrib), _ptr(d_means),
        _ptr(d_log_scales), _ptr(d_quats), _ptr(d_opacity_logits), _ptr(d_sh), _ptr(workspace), _stream(stream)))


def ws_render_train_l2_batch(n, means, log_scales, quats, sh, cams_arr, cfg, num_keys, keys, vals, splats, rect,
                             offsets, tiles_touched, target, key_capacity, ranges, image, t_final, n_contrib, d_means,
                             d_log_scales, d_quats, d_opacity_logits, d_sh, workspace, stream=None):
    _check("ws_render_train_l2_batch", lib().ws_render_train_l2_batch(
        int(n), _ptr(means), _ptr(log_scales), _ptr(quats), _ptr(sh), len(cams_arr), cams_arr, C.byref(cfg),
        _ptr(num_keys), _ptr(keys), _ptr(vals), _ptr(splats), _ptr(rect), _ptr(offsets), _ptr(tiles_touched),
        _ptr(target), int(key_capacity), _ptr(ranges), _ptr(image), _ptr(t_final), _ptr(n_contrib), _ptr(d_means),
        _ptr(d_log_scales), _ptr(d_quats), _ptr(d_opacity_logits), _ptr(d_sh), _ptr(workspace), _stream(stream)))


def frame_buffers(**ptrs) -> FrameBuffers:
    """ws_frame_buffers from device tensors (by field name) and key_capacity."""
    b = FrameBuffers()
    for name, _ in FrameBuffers._fields_:
        if name == "key_capacity":
            b.key_capacity = int(ptrs["key_capacity"])
        else:
            setattr(b, name, _ptr(ptrs[name]))
    return b


def ws_render_frame_host(n, h_scene, cam, cfg, buffers, h_image, stream=None):
    """One frame from host scene arrays (dict of CPU tensors, ideally pinned)
    into a host image tensor (H, W, 3), on `stream`; asynchronous."""
    def hp(t):
        return t.data_ptr() if t.numel() else None
    _check("ws_render_frame_host", lib().ws_render_frame_host(
        int(n), hp(h_scene["means"]), hp(h_scene["log_scales"]), hp(h_scene["quats"]),
        hp(h_scene["opacity_logits"]), hp(h_scene["sh"]), C.byref(cam), C.byref(cfg), C.byref(buffers),
        hp(h_image), _stream(stream)))
