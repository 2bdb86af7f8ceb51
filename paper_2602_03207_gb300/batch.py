"""Batched multi-view rendering and training steps on top of the C ABI.

``BatchRenderer`` owns the buffers of one batch of cameras (uneven
resolutions allowed) of one scene and issues ws_preprocess_batch ->
ws_cull_batch -> ws_sort -> ws_rasterize_batch, and for a training step
ws_image_residual -> ws_rasterize_backward_batch, all on one stream with no
host synchronisation, so a whole step can be captured into a CUDA graph and
replayed. torch only allocates memory and provides streams and graphs.
"""
from __future__ import annotations

import math

import torch

from . import capi
from .render import SCENE_KEYS, config_flags, sort_frame, tile_grid


class BatchRenderer:
    def __init__(self, n, cams, tile=16, digit_bits=9, key_capacity=None, dilation=0.3, guard=1.3, flags=0,
                 device="cuda", sort="segmented", fused=False, persistent=False):
        if not 0 < len(cams) <= capi.ws_batch_max_views():
            raise ValueError(f"1..{capi.ws_batch_max_views()} views per batch")
        self.n, self.V = int(n), len(cams)
        self.cams = list(cams)
        self.cams_arr = capi.camera_array(cams)
        self.fused = bool(fused)
        self.cfg = capi.config(tile=tile, digit_bits=digit_bits, dilation=dilation, guard=guard,
                               flags=config_flags(flags, sort) | (capi.WS_CFG_PERSISTENT if persistent else 0))
        self.tile = tile
        grids = [tile_grid(c["width"], c["height"], tile) for c in cams]
        self.tile_off = [0]
        self.pix_off = [0]
        for (tx, ty), c in zip(grids, cams):
            self.tile_off.append(self.tile_off[-1] + tx * ty)
            self.pix_off.append(self.pix_off[-1] + c["width"] * c["height"])
        self.total_tiles, self.total_pix = self.tile_off[-1], self.pix_off[-1]
        self.end_bit = 31 + max(1, math.ceil(math.log2(self.total_tiles))) if self.total_tiles > 1 else 31
        self.key_capacity = int(key_capacity if key_capacity is not None else max(1024, 2 * self.n * self.V))
        d = torch.device(device)
        vn = max(self.V * self.n, 1)
        cap = max(self.key_capacity, 1)
        self.splats = torch.empty((vn, capi.WS_SPLAT_FLOATS), dtype=torch.float32, device=d)
        self.depth = torch.empty(vn, dtype=torch.float32, device=d)
        self.rect = torch.empty((vn, 4), dtype=torch.int16, device=d)
        self.tiles_touched = torch.empty(vn, dtype=torch.int32, device=d)
        self.offsets = torch.empty(self.V * self.n + 1, dtype=torch.int32, device=d)
        self.keys = torch.empty(cap, dtype=torch.int64, device=d)
        self.vals = torch.empty(cap, dtype=torch.int32, device=d)
        self.keys_alt = torch.empty(cap, dtype=torch.int64, device=d)
        self.vals_alt = torch.empty(cap, dtype=torch.int32, device=d)
        self.num_keys = torch.zeros(4, dtype=torch.int32, device=d)
        self.ranges = torch.empty((max(self.total_tiles, 1), 2), dtype=torch.int32, device=d)
        self.image = torch.empty(self.total_pix * 3, dtype=torch.float32, device=d)
        self.t_final = torch.empty(self.total_pix, dtype=torch.float32, device=d)
        self.n_contrib = torch.empty(self.total_pix, dtype=torch.int32, device=d)
        self.d_image = torch.empty(self.total_pix * 3, dtype=torch.float32, device=d)
        n1 = max(self.n, 1)
        self.grads = {"means": torch.empty((n1, 3), dtype=torch.float32, device=d),
                      "log_scales": torch.empty((n1, 3), dtype=torch.float32, device=d),
                      "quats": torch.empty((n1, 4), dtype=torch.float32, device=d),
                      "opacity_logits": torch.empty(n1, dtype=torch.float32, device=d),
                      "sh": torch.empty((n1, 16, 3), dtype=torch.float32, device=d)}
        nbytes = capi.ws_batch_workspace_bytes(self.n, self.cams_arr, self.key_capacity, self.cfg)
        if nbytes == 0:
            raise ValueError("ws_batch_workspace_bytes rejected the configuration")
        self.workspace = torch.zeros(nbytes, dtype=torch.uint8, device=d)
        self.sorted_in_alt = False

    @property
    def sorted_keys(self):
        return self.keys_alt if self.sorted_in_alt else self.keys

    @property
    def sorted_vals(self):
        return self.vals_alt if self.sorted_in_alt else self.vals

    # views of the view-major splat records (centre hi/lo, conic, sigma, colour)
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
    def preprocess(self, scene, stream=None):
        capi.ws_preprocess_batch(self.n, scene["means"], scene["log_scales"], scene["quats"],
                                 scene["opacity_logits"], scene["sh"], self.cams_arr, self.cfg, self.splats,
                                 self.depth, self.rect, self.tiles_touched, stream)

    def cull(self, stream=None):
        capi.ws_cull_batch(self.n, self.cams_arr, self.cfg, self.tiles_touched, self.rect, self.depth, self.offsets,
                           self.keys, self.vals, self.key_capacity, self.num_keys, self.workspace, stream)

    def sort(self, stream=None):
        sort_frame(self, self.total_tiles, stream)

    def rasterize(self, stream=None):
        capi.ws_rasterize_batch(self.num_keys, self.sorted_keys, self.sorted_vals, self.n, self.splats,
                                self.cams_arr, self.raster_cfg, self.ranges, self.image, self.t_final, self.n_contrib,
                                stream)

    def residual(self, target, stream=None):
        """d_image = image - target (gradient of 1/2 ||image - target||^2)."""
        capi.ws_image_residual(self.total_pix * 3, self.image, target, self.d_image, stream)

    def forward(self, scene, stream=None):
        self.preprocess(scene, stream)
        self.cull(stream)
        self.sort(stream)
        self.rasterize(stream)
        return self.image

    def backward(self, scene, d_image, stream=None):
        g = self.grads
        capi.ws_rasterize_backward_batch(self.n, scene["means"], scene["log_scales"], scene["quats"], scene["sh"],
                                         self.cams_arr, self.cfg, self.splats, self.rect, self.offsets,
                                         self.tiles_touched, self.sorted_vals, self.ranges, self.t_final,
                                         self.n_contrib, d_image, self.key_capacity, g["means"],
                                         g["log_scales"], g["quats"], g["opacity_logits"], g["sh"], self.workspace,
                                         stream)
        return {k: v[:self.n] for k, v in g.items()}

    def step(self, scene, target, stream=None):
        """One training step of 1/2 ||image - target||^2 summed over the views.
        Default: the separate calls (forward, d_image = image - target,
        backward). fused=True (about 1.5 % faster on GB300): pre-processing,
        compaction, sort, then ws_render_train_l2_batch (every (view, tile)
        composited, its residual formed and its backward records written in
        one pass; persistent=True runs that pass as one persistent grid). All
        give the same images and gradients bit for bit."""
        if not self.fused:
            self.forward(scene, stream)
            self.residual(target, stream)
            return self.backward(scene, self.d_image, stream)
        self.preprocess(scene, stream)
        self.cull(stream)
        self.sort(stream)
        return self.train_pass(scene, target, stream)

    def train_pass(self, scene, target, stream=None):
        """The fused pass of a step after the sort (ws_render_train_l2_batch):
        images, L2 residual, backward records and the per-Gaussian gradients
        summed over the views; one persistent grid when persistent=True."""
        g = self.grads
        capi.ws_render_train_l2_batch(self.n, scene["means"], scene["log_scales"], scene["quats"], scene["sh"],
                                      self.cams_arr, self.raster_cfg, self.num_keys, self.sorted_keys, self.sorted_vals,
                                      self.splats, self.rect, self.offsets, self.tiles_touched, target,
                                      self.key_capacity, self.ranges, self.image, self.t_final, self.n_contrib,
                                      g["means"], g["log_scales"], g["quats"], g["opacity_logits"], g["sh"],
                                      self.workspace, stream)
        return {k: v[:self.n] for k, v in g.items()}

    def images(self):
        out = []
        for v, c in enumerate(self.cams):
            a, b = self.pix_off[v] * 3, self.pix_off[v + 1] * 3
            out.append(self.image[a:b].view(c["height"], c["width"], 3))
        return out

    def pack(self, per_view):
        """Packs a list of (H, W, 3) tensors in view order (e.g. targets)."""
        return torch.cat([t.reshape(-1) for t in per_view]).contiguous()

    def capture(self, scene, target):
        """CUDA graph of one training step (forward + residual + backward)."""
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            for _ in range(2):  # warm-up outside the graph
                self.step(scene, target, s)
        torch.cuda.current_stream().wait_stream(s)
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            self.step(scene, target, torch.cuda.current_stream())
        return g

    def check_status(self):
        flags = capi.ws_read_status(self.workspace)
        if flags & capi.WS_FLAG_CAPACITY:
            raise capi.WsError("batch", capi.WS_ERR_CAPACITY)
        return flags

    def key_count(self):
        return int(self.num_keys[0].item())
