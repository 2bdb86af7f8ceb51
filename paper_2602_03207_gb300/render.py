"""Frame orchestration on top of the C ABI.

``Renderer`` owns the device buffers of one resolution and issues the four
C-ABI calls of a frame (ws_preprocess -> ws_cull -> ws_sort -> ws_rasterize)
on the current CUDA stream. It holds no arithmetic of its own: torch only
allocates memory and provides the stream.
"""
from __future__ import annotations

import math

import torch

from . import capi

SCENE_KEYS = ("means", "log_scales", "quats", "opacity_logits", "sh")


def scene_to_device(scene, device="cuda"):
    """numpy scene dict -> contiguous float32 CUDA tensors."""
    out = {}
    for k in SCENE_KEYS:
        out[k] = torch.as_tensor(scene[k], dtype=torch.float32).contiguous().to(device)
    return out


def tile_grid(width, height, tile):
    return (width + tile - 1) // tile, (height + tile - 1) // tile


def key_end_bit(width, height, tile):
    """Keys are (tile id << 31) | depth bits; the sort covers bits [0, end)."""
    tx, ty = tile_grid(width, height, tile)
    tiles = tx * ty
    return 31 + max(1, math.ceil(math.log2(tiles))) if tiles > 1 else 31


SORT_FLAGS = {"segmented": capi.WS_CFG_SORT_SEGMENTED, "lsd": 0, "lookback": capi.WS_CFG_SORT_LOOKBACK}


def with_flags(cfg, extra):
    """A copy of a ws_config with more flag bits set."""
    return capi.Config(cfg.tile, cfg.digit_bits, cfg.dilation, cfg.guard, cfg.flags | int(extra))


def sort_frame(obj, ntiles, stream=None):
    """Sorts obj's pairs. With the segmented sort, ws_sort_tiles also leaves
    the tile ranges in obj.ranges and the rasterisation is told so
    (WS_CFG_RANGES_GIVEN); where that sort does not apply (a single tile, or a
    workspace too small for the segment starts) ws_sort runs and the
    rasterisation finds the ranges itself. Sets obj.sorted_in_alt and
    obj.raster_cfg."""
    if obj.cfg.flags & capi.WS_CFG_SORT_SEGMENTED and getattr(obj, "_tile_sort", True):
        try:
            obj.sorted_in_alt = capi.ws_sort_tiles(obj.num_keys, obj.key_capacity, obj.end_bit, obj.keys, obj.vals,
                                                   obj.keys_alt, obj.vals_alt, obj.cfg, obj.workspace, obj.ranges,
                                                   ntiles, stream)
            obj.raster_cfg = with_flags(obj.cfg, capi.WS_CFG_RANGES_GIVEN)
            return
        except capi.WsError as e:
            if e.status != capi.WS_ERR_UNSUPPORTED:
                raise
            obj._tile_sort = False
    obj.sorted_in_alt = capi.ws_sort(obj.num_keys, obj.key_capacity, 0, obj.end_bit, obj.keys, obj.vals,
                                     obj.keys_alt, obj.vals_alt, obj.cfg, obj.workspace, stream)
    obj.raster_cfg = obj.cfg


def config_flags(flags, sort):
    """ws_config.flags for the user's flags and a sort variant: "segmented"
    (partition by tile, then each tile's depths on chip), "lsd" (full-key
    passes) or "lookback" (single-sweep look-back passes). All three give
    the same sorted pairs."""
    if sort not in SORT_FLAGS:
        raise ValueError(f"sort must be one of {sorted(SORT_FLAGS)}, got {sort!r}")
    return int(flags) | SORT_FLAGS[sort]


class Renderer:
    """Buffers and calls for frames of a fixed (n, width, height, tile)."""

    def __init__(self, n, width, height, tile=16, digit_bits=8, key_capacity=None, dilation=0.3,
                 guard=1.3, flags=0, device="cuda", sort="segmented", packed=False, fused_cull=False):
        self.n, self.width, self.height = int(n), int(width), int(height)
        self.fused_cull = bool(fused_cull)  # forward(): ws_cull_sort_tiles instead of ws_cull + the sort
        self.cfg = capi.config(tile=tile, digit_bits=digit_bits, dilation=dilation, guard=guard,
                               flags=config_flags(flags, sort))
        self.tile = tile
        self.tx, self.ty = tile_grid(width, height, tile)
        self.key_capacity = int(key_capacity if key_capacity is not None else max(1024, 4 * self.n))
        self.end_bit = key_end_bit(width, height, tile)
        d = torch.device(device)
        n1 = max(self.n, 1)
        cap = max(self.key_capacity, 1)
        self.splats = torch.empty((n1, capi.WS_SPLAT_FLOATS), dtype=torch.float32, device=d)
        self.depth = torch.empty(n1, dtype=torch.float32, device=d)
        self.rect = torch.empty((n1, 4), dtype=torch.int16, device=d)       # uint16 payload
        self.tiles_touched = torch.empty(n1, dtype=torch.int32, device=d)   # uint32 payload
        self.offsets = torch.empty(self.n + 1, dtype=torch.int32, device=d)
        self.keys = torch.empty(cap, dtype=torch.int64, device=d)           # uint64 payload
        self.vals = torch.empty(cap, dtype=torch.int32, device=d)
        self.keys_alt = torch.empty(cap, dtype=torch.int64, device=d)
        self.vals_alt = torch.empty(cap, dtype=torch.int32, device=d)
        self.num_keys = torch.zeros(4, dtype=torch.int32, device=d)
        self.ranges = torch.empty((self.tx * self.ty, 2), dtype=torch.int32, device=d)
        self.image = torch.empty((height, width, 3), dtype=torch.float32, device=d)
        self.t_final = torch.empty((height, width), dtype=torch.float32, device=d)
        self.n_contrib = torch.empty((height, width), dtype=torch.int32, device=d)
        # packed-record variant (ws_preprocess_packed / ws_rasterize_packed)
        self.packed = bool(packed)
        if self.packed:
            self.mean2d_p = torch.empty((n1, 2), dtype=torch.float32, device=d)
            self.axes = torch.empty((n1, 2), dtype=torch.int32, device=d)      # 2 x (2 binary16)
            self.rgba = torch.empty(n1, dtype=torch.int32, device=d)           # RGBA8
        self._cam_probe = None
        self.workspace = None
        self.sorted_in_alt = False

    def _ensure_workspace(self, cam):
        if self.workspace is None:
            nbytes = capi.ws_workspace_bytes(self.n, self.key_capacity, cam, self.cfg)
            if nbytes == 0:
                raise ValueError("ws_workspace_bytes rejected the configuration")
            self.workspace = torch.zeros(nbytes, dtype=torch.uint8, device=self.image.device)

    # views of the splat record (centre hi/lo, conic, sigma, colour)
    @property
    def mean2d(self):
        return self.splats[:, 0:4]

    @property
    def conic(self):
        return self.splats[:, 4:7]

    @property
    def opacity(self):
        return self.splats[:, 7]

    @property
    def rgb(self):
        return self.splats[:, 8:11]

    # ------------------------------------------------------------ stages
    def preprocess(self, scene, cam, stream=None):
        if self.packed:
            capi.ws_preprocess_packed(self.n, scene["means"], scene["log_scales"], scene["quats"],
                                      scene["opacity_logits"], scene["sh"], cam, self.cfg, self.mean2d_p,
                                      self.axes, self.rgba, self.depth, self.rect, self.tiles_touched, stream)
            return
        capi.ws_preprocess(self.n, scene["means"], scene["log_scales"], scene["quats"],
                           scene["opacity_logits"], scene["sh"], cam, self.cfg, self.splats, self.depth, self.rect,
                           self.tiles_touched, stream)

    def cull(self, cam, stream=None):
        self._ensure_workspace(cam)
        capi.ws_cull(self.n, self.tiles_touched, self.rect, self.depth, cam, self.cfg, self.offsets,
                     self.keys, self.vals, self.key_capacity, self.num_keys, self.workspace, stream)

    def sort(self, stream=None):
        sort_frame(self, self.tx * self.ty, stream)

    def _cull_and_sort(self, cam, stream=None):
        if self.fused_cull:
            self.cull_sort(cam, stream)
        else:
            self.cull(cam, stream)
            self.sort(stream)

    def cull_sort(self, cam, stream=None):
        """cull() then sort(), as one call where it applies: with the
        segmented sort, ws_cull_sort_tiles writes each pair straight into the
        sort's first partition (the same results, one pass fewer over the
        pairs; on GB300 no faster than the two calls, which forward() takes
        unless the renderer was made with fused_cull=True); otherwise the
        two calls."""
        self._ensure_workspace(cam)
        if self.cfg.flags & capi.WS_CFG_SORT_SEGMENTED and getattr(self, "_fused_cull", True):
            try:
                self.sorted_in_alt = capi.ws_cull_sort_tiles(
                    self.n, self.tiles_touched, self.rect, self.depth, cam, self.cfg, self.offsets, self.keys,
                    self.vals, self.keys_alt, self.vals_alt, self.key_capacity, self.num_keys, self.ranges,
                    self.workspace, stream)
                self.raster_cfg = with_flags(self.cfg, capi.WS_CFG_RANGES_GIVEN)
                return
            except capi.WsError as e:
                if e.status != capi.WS_ERR_UNSUPPORTED:
                    raise
                self._fused_cull = False
        self.cull(cam, stream)
        self.sort(stream)

    @property
    def sorted_keys(self):
        return self.keys_alt if self.sorted_in_alt else self.keys

    @property
    def sorted_vals(self):
        return self.vals_alt if self.sorted_in_alt else self.vals

    def rasterize(self, cam, stream=None):
        if self.packed:
            capi.ws_rasterize_packed(self.num_keys, self.sorted_keys, self.sorted_vals, self.mean2d_p, self.axes,
                                     self.rgba, cam, self.raster_cfg, self.ranges, self.image, self.t_final,
                                     self.n_contrib, stream)
            return
        capi.ws_rasterize(self.num_keys, self.sorted_keys, self.sorted_vals, self.splats, cam, self.raster_cfg,
                          self.ranges, self.image, self.t_final, self.n_contrib, stream)

    def forward(self, scene, cam_dict, stream=None):
        """One frame; returns the image tensor (H, W, 3). Asynchronous."""
        cam = capi.camera(cam_dict)
        if cam.width != self.width or cam.height != self.height:
            raise ValueError("camera resolution differs from the renderer's")
        self.preprocess(scene, cam, stream)
        self._cull_and_sort(cam, stream)
        self.rasterize(cam, stream)
        return self.image

    def forward_quads(self, scene, cam_dict, stream=None):
        """One frame through the paper's own design (ws_render_quads: global
        depth sort, opacity-sized quads, back-to-front "over"); image and
        t_final as forward(). Asynchronous."""
        if self.packed:
            raise ValueError("the quad path takes the float pre-processing outputs")
        cam = capi.camera(cam_dict)
        self.preprocess(scene, cam, stream)
        if getattr(self, "quad_workspace", None) is None:
            nbytes = capi.ws_quads_workspace_bytes(self.n, self.key_capacity, cam, self.cfg)
            if nbytes == 0:
                raise ValueError("ws_quads_workspace_bytes rejected the configuration")
            self.quad_workspace = torch.zeros(nbytes, dtype=torch.uint8, device=self.image.device)
        capi.ws_render_quads(self.n, self.splats, self.depth, self.tiles_touched, cam, self.cfg,
                             self.key_capacity, self.keys, self.vals, self.keys_alt, self.vals_alt, self.num_keys,
                             self.image, self.t_final, self.quad_workspace, stream)
        return self.image

    def check_quads_status(self, stream=None):
        flags = capi.ws_read_status(self.quad_workspace, clear=False, stream=stream)
        if flags & capi.WS_FLAG_CAPACITY:
            raise capi.WsError("quads", capi.WS_ERR_CAPACITY)
        return flags

    def backward(self, scene, cam_dict, d_image, stream=None):
        """Gradients of a loss w.r.t. the Gaussians for the frame last
        rendered by forward() with the same scene and camera; d_image is
        dL/dimage (H, W, 3). Returns a dict of gradient tensors."""
        if self.packed:
            raise ValueError("the packed-record variant renders only (no backward)")
        cam = capi.camera(cam_dict)
        d = self.image.device
        n1 = max(self.n, 1)
        g = {"means": torch.empty((n1, 3), dtype=torch.float32, device=d),
             "log_scales": torch.empty((n1, 3), dtype=torch.float32, device=d),
             "quats": torch.empty((n1, 4), dtype=torch.float32, device=d),
             "opacity_logits": torch.empty(n1, dtype=torch.float32, device=d),
             "sh": torch.empty((n1, 16, 3), dtype=torch.float32, device=d)}
        d_image = d_image.contiguous()
        capi.ws_rasterize_backward(self.n, scene["means"], scene["log_scales"], scene["quats"],
                                   scene["opacity_logits"], scene["sh"], cam, self.cfg, self.splats, self.rect,
                                   self.offsets, self.tiles_touched,
                                   self.sorted_vals, self.ranges, self.t_final, self.n_contrib, d_image,
                                   self.key_capacity, g["means"], g["log_scales"], g["quats"],
                                   g["opacity_logits"], g["sh"], self.workspace, stream)
        return {k: v[:self.n] for k, v in g.items()}

    def train_step_l2(self, scene, cam_dict, target, stream=None):
        """One training step of L = 1/2 ||image - target||^2 in fused form
        (ws_render_train_l2 after the pre-processing, compaction and sort):
        the same image and gradients as forward() + ws_image_residual +
        backward(), in fewer launches. Returns the gradient dict."""
        if self.packed:
            raise ValueError("the packed-record variant renders only (no backward)")
        cam = capi.camera(cam_dict)
        self.preprocess(scene, cam, stream)
        self._cull_and_sort(cam, stream)
        return self.train_pass_l2(scene, cam_dict, target, stream)

    def train_pass_l2(self, scene, cam_dict, target, stream=None):
        """The fused pass of train_step_l2 alone (ws_render_train_l2), on the
        pairs this renderer has sorted for the same scene and camera."""
        cam = capi.camera(cam_dict)
        g = self._grads()
        capi.ws_render_train_l2(self.n, scene["means"], scene["log_scales"], scene["quats"], scene["sh"], cam,
                                self.raster_cfg, self.num_keys, self.sorted_keys, self.sorted_vals, self.splats, self.rect,
                                self.offsets, self.tiles_touched, target.contiguous(), self.key_capacity,
                                self.ranges, self.image, self.t_final, self.n_contrib, g["means"], g["log_scales"],
                                g["quats"], g["opacity_logits"], g["sh"], self.workspace, stream)
        return {k: v[:self.n] for k, v in g.items()}

    def _grads(self):
        if getattr(self, "grads", None) is None:
            d = self.image.device
            n1 = max(self.n, 1)
            self.grads = {"means": torch.empty((n1, 3), dtype=torch.float32, device=d),
                          "log_scales": torch.empty((n1, 3), dtype=torch.float32, device=d),
                          "quats": torch.empty((n1, 4), dtype=torch.float32, device=d),
                          "opacity_logits": torch.empty(n1, dtype=torch.float32, device=d),
                          "sh": torch.empty((n1, 16, 3), dtype=torch.float32, device=d)}
        return self.grads

    def check_status(self, stream=None):
        """Synchronises and raises if the frame overflowed its key capacity."""
        flags = capi.ws_read_status(self.workspace, clear=False, stream=stream)
        if flags & capi.WS_FLAG_CAPACITY:
            raise capi.WsError("frame", capi.WS_ERR_CAPACITY)
        return flags

    def key_count(self):
        return int(self.num_keys[0].item())

    def total_pairs(self):
        return int(self.offsets[self.n].item()) & 0xFFFFFFFF


class FramePipeline:
    """Frames whose scene and image live in host memory, each rendered by one
    C-ABI call (ws_render_frame_host: the scene's host -> device copies, the
    four stages and the image's device -> host copy, on one stream). Each of
    `slots` slots owns a Renderer, the device copy of the scene and a stream,
    and frames go to the slots in turn, so frame i+1's upload overlaps frame
    i's render and read-back and a stream of frames runs at the pace of the
    host-device link rather than upload + render + read-back in series. A
    slot's next frame follows its previous one on its stream. Everything is
    asynchronous; synchronize() waits for all frames and checks each
    renderer's status."""

    def __init__(self, n, width, height, slots=2, device="cuda", **renderer_kw):
        self.device = torch.device(device)
        self.n = int(n)
        self.slots = []
        for _ in range(int(slots)):
            r = Renderer(n, width, height, device=self.device, **renderer_kw)
            scene = {k: torch.empty(shape, dtype=torch.float32, device=self.device)
                     for k, shape in (("means", (max(n, 1), 3)), ("log_scales", (max(n, 1), 3)),
                                      ("quats", (max(n, 1), 4)), ("opacity_logits", (max(n, 1),)),
                                      ("sh", (max(n, 1), 16, 3)))}
            self.slots.append({"r": r, "scene": scene, "stream": torch.cuda.Stream(self.device), "buf": None})
        self.count = 0

    def streams(self):
        return [s["stream"] for s in self.slots]

    def submit(self, host_scene, cam_dict, host_image):
        """Queue one frame: host_scene (dict of CPU float32 tensors in the
        input layouts, ideally pinned), cam_dict, host_image (a CPU float32
        tensor (H, W, 3), ideally pinned). Returns at once."""
        s = self.slots[self.count % len(self.slots)]
        self.count += 1
        r = s["r"]
        cam = capi.camera(cam_dict)
        if s["buf"] is None:
            r._ensure_workspace(cam)
            s["buf"] = capi.frame_buffers(
                **s["scene"], splats=r.splats, depth=r.depth, rect=r.rect, tiles_touched=r.tiles_touched,
                offsets=r.offsets, keys=r.keys, keys_alt=r.keys_alt, vals=r.vals, vals_alt=r.vals_alt,
                num_keys=r.num_keys, ranges=r.ranges, image=r.image, t_final=r.t_final, n_contrib=r.n_contrib,
                workspace=r.workspace, key_capacity=r.key_capacity)
        capi.ws_render_frame_host(self.n, host_scene, cam, r.cfg, s["buf"], host_image, s["stream"])

    def synchronize(self):
        torch.cuda.synchronize(self.device)
        for s in self.slots:
            s["r"].check_status()


def render(scene, cam_dict, tile=16, digit_bits=8, key_capacity=None, flags=0, sort="segmented"):
    """Render one frame of a device scene dict; returns (image, renderer).

    Raises when the pair list overflows the key capacity (after a sync)."""
    n = scene["means"].shape[0]
    r = Renderer(n, cam_dict["width"], cam_dict["height"], tile=tile, digit_bits=digit_bits,
                 key_capacity=key_capacity, flags=flags, device=scene["means"].device, sort=sort)
    img = r.forward(scene, cam_dict)
    r.check_status()
    return img, r


class RenderFunction(torch.autograd.Function):
    """Differentiable frame: image = render(means, log_scales, quats,
    opacity_logits, sh). The renderer's buffers hold the frame's
    intermediates between forward and backward, so one renderer serves one
    frame in flight at a time.

    Forward and backward only enqueue work on the current stream: nothing
    synchronises the host, so a whole training step can be captured in a
    CUDA graph. The capacity check is the caller's: renderer.check_status()
    (which synchronises) after the step raises if the frame's pairs
    overflowed the key capacity, in which case the step's image and
    gradients are incomplete."""

    @staticmethod
    def forward(ctx, means, log_scales, quats, opacity_logits, sh, renderer, cam_dict):
        scene = {"means": means.contiguous(), "log_scales": log_scales.contiguous(),
                 "quats": quats.contiguous(), "opacity_logits": opacity_logits.contiguous(),
                 "sh": sh.contiguous()}
        img = renderer.forward(scene, cam_dict)
        ctx.renderer, ctx.cam, ctx.scene = renderer, cam_dict, scene
        return img.clone()

    @staticmethod
    def backward(ctx, d_image):
        g = ctx.renderer.backward(ctx.scene, ctx.cam, d_image)
        return g["means"], g["log_scales"], g["quats"], g["opacity_logits"], g["sh"], None, None


def render_differentiable(params, renderer, cam_dict):
    """params: dict of leaf tensors (means, log_scales, quats,
    opacity_logits, sh); returns the image with autograd attached.
    Asynchronous; check renderer.check_status() after the step."""
    return RenderFunction.apply(params["means"], params["log_scales"], params["quats"],
                                params["opacity_logits"], params["sh"], renderer, cam_dict)
