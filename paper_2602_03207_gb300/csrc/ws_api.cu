// extern "C" entry points of websplat.h: host-side argument checks, frame
// constants and workspace layout; every launch goes to the kernels in
// ws_preprocess.cu, ws_cull.cu, ws_sort.cu and ws_raster.cu.
#include <cmath>
#include <cstring>

#include "websplat.h"
#include "ws_common.cuh"
#include "ws_kernels.cuh"

namespace {

using ws::Frame;

bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

bool valid_tile(int t) { return t == 8 || t == 16 || t == 32; }

bool valid_camera(const ws_camera* c) {
    if (!c) return false;
    if (c->width <= 0 || c->height <= 0 || c->width > 65535 * 8 || c->height > 65535 * 8) return false;
    if (!(c->fx > 0.f) || !(c->fy > 0.f) || !(c->znear >= 0.f)) return false;
    for (int i = 0; i < 12; ++i)
        if (!std::isfinite(c->viewmat[i])) return false;
    return std::isfinite(c->cx) && std::isfinite(c->cy);
}

bool valid_config(const ws_config* g) {
    return g && valid_tile(g->tile) && g->dilation >= 0.f && g->guard > 0.f;
}

Frame make_frame(const ws_camera* c, const ws_config* g) {
    Frame f;
    for (int r = 0; r < 3; ++r) {
        for (int k = 0; k < 3; ++k) f.R[3 * r + k] = c->viewmat[4 * r + k];
        f.t[r] = c->viewmat[4 * r + 3];
    }
    for (int k = 0; k < 3; ++k)
        f.campos[k] = -(f.R[k] * f.t[0] + f.R[3 + k] * f.t[1] + f.R[6 + k] * f.t[2]);
    f.fx = c->fx;
    f.fy = c->fy;
    f.cx = c->cx;
    f.cy = c->cy;
    f.znear = c->znear;
    f.limx = g->guard * 0.5f * (float)c->width / c->fx;
    f.limy = g->guard * 0.5f * (float)c->height / c->fy;
    f.dilation = g->dilation;
    for (int k = 0; k < 3; ++k) f.bg[k] = c->bg[k];
    f.W = c->width;
    f.H = c->height;
    f.TS = g->tile;
    f.TX = (c->width + g->tile - 1) / g->tile;
    f.TY = (c->height + g->tile - 1) / g->tile;
    f.flags = g->flags;
    return f;
}

size_t align_up(size_t v) { return (v + 255) & ~size_t(255); }

// Workspace layout: [status | sort scratch | pair records | compaction
// scratch]. The first three depend only on the key capacity (the sort region
// is sized for the widest supported digit, so any digit width fits), so
// ws_sort and ws_rasterize_backward find their regions without knowing n.
constexpr int kMaxDigitBits = 11;

struct Layout {
    size_t status, sort, bwd, cull, total;
};

Layout layout(int64_t n, int64_t cap) {
    Layout L;
    L.status = 0;
    L.sort = align_up(ws::kStatusBytes);
    size_t sort_bytes = ws::sort_scratch_bytes(cap, kMaxDigitBits);
    if (ws::sort_lookback_scratch_bytes(cap) > sort_bytes) sort_bytes = ws::sort_lookback_scratch_bytes(cap);
    if (ws::sort_segmented_scratch_bytes(cap) > sort_bytes) sort_bytes = ws::sort_segmented_scratch_bytes(cap);
    L.bwd = L.sort + align_up(sort_bytes);
    L.cull = L.bwd + align_up(ws::backward_scratch_bytes(cap));
    L.total = L.cull + align_up(ws::cull_scratch_bytes(n));
    return L;
}

ws_status cuda_status(cudaError_t e) { return e == cudaSuccess ? WS_OK : WS_ERR_CUDA; }

// Host-side table of a batch's cameras: per-view frame constants and the
// global tile / pixel numbering. Returns false for invalid arguments.
bool make_table(int32_t views, const ws_camera* cams, const ws_config* cfg, ws::FrameTable& ft) {
    if (views <= 0 || views > ws::kMaxViews || !cams || !valid_config(cfg)) return false;
    ft.views = views;
    ft.tile_off[0] = 0;
    ft.pix_off[0] = 0;
    for (int v = 0; v < views; ++v) {
        if (!valid_camera(cams + v)) return false;
        ft.f[v] = make_frame(cams + v, cfg);
        if (ft.f[v].TX > 65535 || ft.f[v].TY > 65535) return false;
        const uint64_t t = (uint64_t)ft.tile_off[v] + (uint64_t)ft.f[v].TX * ft.f[v].TY;
        if (t >= (uint64_t(1) << 32)) return false;
        ft.tile_off[v + 1] = (uint32_t)t;
        ft.pix_off[v + 1] = ft.pix_off[v] + (uint64_t)cams[v].width * cams[v].height;
    }
    for (int v = views; v < ws::kMaxViews; ++v) ft.tile_off[v + 1] = ft.tile_off[views];
    return true;
}

ws::ViewGrid make_grid(const ws::FrameTable& ft) {
    ws::ViewGrid g;
    g.views = ft.views;
    for (int v = 0; v <= ws::kMaxViews; ++v) g.tile_off[v] = ft.tile_off[v];
    for (int v = 0; v < ws::kMaxViews; ++v) g.tiles_x[v] = v < ft.views ? (uint32_t)ft.f[v].TX : 0u;
    return g;
}

}  // namespace

extern "C" {

int32_t ws_abi_version(void) { return WS_ABI_VERSION; }

const char* ws_status_string(ws_status s) {
    switch (s) {
        case WS_OK: return "ok";
        case WS_ERR_INVALID_ARG: return "invalid argument";
        case WS_ERR_CUDA: return "CUDA error";
        case WS_ERR_CAPACITY: return "key capacity exceeded";
        case WS_ERR_TIMEOUT: return "bounded wait timed out";
        case WS_ERR_UNSUPPORTED: return "unsupported configuration";
        default: return "unknown status";
    }
}

size_t ws_workspace_bytes(int64_t n, int64_t key_capacity, const ws_camera* cam, const ws_config* cfg) {
    if (n < 0 || key_capacity < 0 || key_capacity >= (int64_t(1) << 31)) return 0;
    if (!valid_camera(cam) || !valid_config(cfg) || !ws::sort_digit_supported(cfg->digit_bits)) return 0;
    // one view: the layout, then the fused compaction's digit counts
    return layout(n, key_capacity).total + align_up(ws::cull_partition_scratch_bytes(n));
}

ws_status ws_preprocess(int64_t n, const float* means, const float* log_scales, const float* quats,
                        const float* opacity_logits, const float* sh, const ws_camera* cam,
                        const ws_config* cfg, float* splats, float* depth, uint16_t* rect,
                        uint32_t* tiles_touched, void* stream) {
    if (n < 0 || n >= (int64_t(1) << 32) || !valid_camera(cam) || !valid_config(cfg)) return WS_ERR_INVALID_ARG;
    if (n == 0) return WS_OK;
    const void* ptrs[] = {means, log_scales, quats, opacity_logits, sh, splats, depth, rect, tiles_touched};
    for (const void* p : ptrs)
        if (!p || !aligned16(p)) return WS_ERR_INVALID_ARG;
    const Frame f = make_frame(cam, cfg);
    if (f.TX > 65535 || f.TY > 65535) return WS_ERR_UNSUPPORTED;
    return cuda_status(ws::launch_preprocess(n, means, log_scales, quats, opacity_logits, sh, f,
                                             splats, depth, rect, tiles_touched,
                                             static_cast<cudaStream_t>(stream)));
}

ws_status ws_cull(int64_t n, const uint32_t* tiles_touched, const uint16_t* rect, const float* depth,
                  const ws_camera* cam, const ws_config* cfg, uint32_t* offsets, uint64_t* keys,
                  uint32_t* vals, int64_t key_capacity, uint32_t* num_keys, void* workspace,
                  void* stream) {
    if (n < 0 || n >= (int64_t(1) << 32) || key_capacity < 0 || key_capacity >= (int64_t(1) << 31))
        return WS_ERR_INVALID_ARG;
    if (!valid_camera(cam) || !valid_config(cfg) || !ws::sort_digit_supported(cfg->digit_bits))
        return WS_ERR_INVALID_ARG;
    const void* ptrs[] = {offsets, num_keys, workspace};
    for (const void* p : ptrs)
        if (!p || !aligned16(p)) return WS_ERR_INVALID_ARG;
    if (n > 0) {
        const void* in[] = {tiles_touched, rect, depth};
        for (const void* p : in)
            if (!p || !aligned16(p)) return WS_ERR_INVALID_ARG;
    }
    if (key_capacity > 0 && (!keys || !vals || !aligned16(keys) || !aligned16(vals))) return WS_ERR_INVALID_ARG;
    const Frame f = make_frame(cam, cfg);
    const Layout L = layout(n, key_capacity);
    char* ws_base = static_cast<char*>(workspace);
    uint32_t* status = reinterpret_cast<uint32_t*>(ws_base + L.status);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    return cuda_status(ws::launch_cull(n, tiles_touched, rect, depth, f, offsets, keys, vals,
                                       key_capacity, num_keys, status, ws_base + L.cull, s));
}

ws_status ws_cull_sort_tiles(int64_t n, const uint32_t* tiles_touched, const uint16_t* rect, const float* depth,
                             const ws_camera* cam, const ws_config* cfg, uint32_t* offsets, uint64_t* keys,
                             uint32_t* vals, uint64_t* keys_alt, uint32_t* vals_alt, int64_t key_capacity,
                             uint32_t* num_keys, uint32_t* ranges, void* workspace, int32_t* result_in_alt,
                             void* stream) {
    if (n < 0 || n >= (int64_t(1) << 32) || key_capacity < 0 || key_capacity >= (int64_t(1) << 31) ||
        !result_in_alt)
        return WS_ERR_INVALID_ARG;
    if (!valid_camera(cam) || !valid_config(cfg) || !ws::sort_digit_supported(cfg->digit_bits))
        return WS_ERR_INVALID_ARG;
    const void* ptrs[] = {offsets, num_keys, workspace, ranges};
    for (const void* p : ptrs)
        if (!p || !aligned16(p)) return WS_ERR_INVALID_ARG;
    if (n > 0) {
        const void* in[] = {tiles_touched, rect, depth};
        for (const void* p : in)
            if (!p || !aligned16(p)) return WS_ERR_INVALID_ARG;
    }
    if (key_capacity > 0) {
        const void* kp[] = {keys, vals, keys_alt, vals_alt};
        for (const void* p : kp)
            if (!p || !aligned16(p)) return WS_ERR_INVALID_ARG;
    }
    const Frame f = make_frame(cam, cfg);
    const int64_t tiles = (int64_t)f.TX * f.TY;
    int end_bit = 31;
    while ((int64_t(1) << (end_bit - 31)) < tiles) ++end_bit;
    if (end_bit == 31) end_bit = 32;
    const int digit = ws::sort_segmented_first_digit(end_bit, cfg->digit_bits);
    if (!ws::sort_segmented_supported(key_capacity, 0, end_bit) || !ws::cull_partition_supported(digit))
        return WS_ERR_UNSUPPORTED;
    const Layout L = layout(n, key_capacity);
    char* ws_base = static_cast<char*>(workspace);
    uint32_t* status = reinterpret_cast<uint32_t*>(ws_base + L.status);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaError_t e = ws::launch_cull_partition(n, tiles_touched, rect, depth, f, digit, offsets, keys, vals,
                                              key_capacity, num_keys, status, ws_base + L.cull, ws_base + L.total, s);
    if (e != cudaSuccess) return WS_ERR_CUDA;
    int in_alt = 0;
    e = ws::launch_sort_segmented(num_keys, key_capacity, 0, end_bit, cfg->digit_bits, keys, vals, keys_alt,
                                  vals_alt, ws_base + L.sort, &in_alt, s, ranges, (uint32_t)tiles, true);
    *result_in_alt = in_alt;
    return cuda_status(e);
}

ws_status ws_sort(const uint32_t* num_keys, int64_t key_capacity, int32_t begin_bit, int32_t end_bit,
                  uint64_t* keys, uint32_t* vals, uint64_t* keys_alt, uint32_t* vals_alt,
                  const ws_config* cfg, void* workspace, int32_t* result_in_alt, void* stream) {
    if (!cfg || !ws::sort_digit_supported(cfg->digit_bits)) return WS_ERR_UNSUPPORTED;
    if (key_capacity < 0 || key_capacity >= (int64_t(1) << 31) || begin_bit < 0 || end_bit > 64 ||
        begin_bit >= end_bit || !result_in_alt)
        return WS_ERR_INVALID_ARG;
    const void* ptrs[] = {num_keys, workspace};
    for (const void* p : ptrs)
        if (!p || !aligned16(p)) return WS_ERR_INVALID_ARG;
    if (key_capacity > 0) {
        const void* kp[] = {keys, vals, keys_alt, vals_alt};
        for (const void* p : kp)
            if (!p || !aligned16(p)) return WS_ERR_INVALID_ARG;
    }
    char* ws_base = static_cast<char*>(workspace);
    int in_alt = 0;
    cudaError_t e;
    if (cfg->flags & WS_CFG_SORT_LOOKBACK) {
        if (!ws::sort_lookback_supported(cfg->digit_bits, begin_bit, end_bit)) return WS_ERR_UNSUPPORTED;
        e = ws::launch_sort_lookback(num_keys, key_capacity, begin_bit, end_bit, cfg->digit_bits, keys, vals,
                                     keys_alt, vals_alt, ws_base + layout(0, key_capacity).sort,
                                     reinterpret_cast<uint32_t*>(ws_base), -1, &in_alt,
                                     static_cast<cudaStream_t>(stream));
    } else if ((cfg->flags & WS_CFG_SORT_SEGMENTED) &&
               ws::sort_segmented_supported(key_capacity, begin_bit, end_bit)) {
        e = ws::launch_sort_segmented(num_keys, key_capacity, begin_bit, end_bit, cfg->digit_bits, keys, vals,
                                      keys_alt, vals_alt,
                                      ws_base + layout(0, key_capacity).sort, &in_alt,
                                      static_cast<cudaStream_t>(stream));
    } else {
        e = ws::launch_sort(num_keys, key_capacity, begin_bit, end_bit, cfg->digit_bits, keys, vals, keys_alt,
                            vals_alt, ws_base + layout(0, key_capacity).sort, &in_alt,
                            static_cast<cudaStream_t>(stream));
    }
    *result_in_alt = in_alt;
    return cuda_status(e);
}

ws_status ws_sort_tiles(const uint32_t* num_keys, int64_t key_capacity, int32_t end_bit, uint64_t* keys,
                        uint32_t* vals, uint64_t* keys_alt, uint32_t* vals_alt, const ws_config* cfg,
                        void* workspace, uint32_t* ranges, int64_t ntiles, int32_t* result_in_alt, void* stream) {
    if (!cfg || !ws::sort_digit_supported(cfg->digit_bits)) return WS_ERR_UNSUPPORTED;
    if (key_capacity < 0 || key_capacity >= (int64_t(1) << 31) || end_bit > 64 || end_bit < 1 || !result_in_alt ||
        ntiles < 0)
        return WS_ERR_INVALID_ARG;
    if (!ws::sort_segmented_supported(key_capacity, 0, end_bit)) return WS_ERR_UNSUPPORTED;
    if (ntiles > (int64_t(1) << (end_bit - 31))) return WS_ERR_INVALID_ARG;
    const void* ptrs[] = {num_keys, workspace, ranges};
    for (const void* p : ptrs)
        if (!p || !aligned16(p)) return WS_ERR_INVALID_ARG;
    if (key_capacity > 0) {
        const void* kp[] = {keys, vals, keys_alt, vals_alt};
        for (const void* p : kp)
            if (!p || !aligned16(p)) return WS_ERR_INVALID_ARG;
    }
    char* ws_base = static_cast<char*>(workspace);
    int in_alt = 0;
    const cudaError_t e = ws::launch_sort_segmented(num_keys, key_capacity, 0, end_bit, cfg->digit_bits, keys, vals,
                                                    keys_alt, vals_alt, ws_base + layout(0, key_capacity).sort,
                                                    &in_alt, static_cast<cudaStream_t>(stream), ranges,
                                                    (uint32_t)ntiles);
    *result_in_alt = in_alt;
    return cuda_status(e);
}

ws_status ws_sort_test_stalled_tile(const uint32_t* num_keys, int64_t key_capacity, int32_t begin_bit,
                                    int32_t end_bit, uint64_t* keys, uint32_t* vals, uint64_t* keys_alt,
                                    uint32_t* vals_alt, const ws_config* cfg, void* workspace, int32_t stalled_tile,
                                    int32_t* result_in_alt, void* stream) {
    if (!cfg || !ws::sort_lookback_supported(cfg->digit_bits, begin_bit, end_bit)) return WS_ERR_UNSUPPORTED;
    if (key_capacity <= 0 || key_capacity >= (int64_t(1) << 31) || begin_bit < 0 || end_bit > 64 ||
        begin_bit >= end_bit || !result_in_alt || stalled_tile < 0)
        return WS_ERR_INVALID_ARG;
    const void* ptrs[] = {num_keys, workspace, keys, vals, keys_alt, vals_alt};
    for (const void* p : ptrs)
        if (!p || !aligned16(p)) return WS_ERR_INVALID_ARG;
    char* ws_base = static_cast<char*>(workspace);
    int in_alt = 0;
    cudaError_t e = ws::launch_sort_lookback(num_keys, key_capacity, begin_bit, end_bit, cfg->digit_bits, keys, vals,
                                             keys_alt, vals_alt, ws_base + layout(0, key_capacity).sort,
                                             reinterpret_cast<uint32_t*>(ws_base), stalled_tile, &in_alt,
                                             static_cast<cudaStream_t>(stream));
    *result_in_alt = in_alt;
    return cuda_status(e);
}

int64_t ws_sort_noalloc_max_keys(void) { return ws::sort_noalloc_max_keys(); }

ws_status ws_sort_noalloc(const uint32_t* num_keys, int64_t key_capacity, int32_t begin_bit, int32_t end_bit,
                          uint64_t* keys, uint32_t* vals, uint64_t* keys_alt, uint32_t* vals_alt,
                          int32_t digit_bits, int32_t* result_in_alt, void* stream) {
    if (!ws::sort_digit_supported(digit_bits) || digit_bits > 8) return WS_ERR_UNSUPPORTED;
    if (key_capacity < 0 || key_capacity > ws::sort_noalloc_max_keys() || begin_bit < 0 || end_bit > 64 ||
        begin_bit >= end_bit || !result_in_alt)
        return WS_ERR_INVALID_ARG;
    if (!num_keys || !aligned16(num_keys)) return WS_ERR_INVALID_ARG;
    if (key_capacity > 0) {
        const void* kp[] = {keys, vals, keys_alt, vals_alt};
        for (const void* p : kp)
            if (!p || !aligned16(p)) return WS_ERR_INVALID_ARG;
    }
    int in_alt = 0;
    cudaError_t e = ws::launch_sort_noalloc(num_keys, key_capacity, begin_bit, end_bit, digit_bits, keys, vals,
                                            keys_alt, vals_alt, &in_alt, static_cast<cudaStream_t>(stream));
    *result_in_alt = in_alt;
    return cuda_status(e);
}

ws_status ws_rasterize(const uint32_t* num_keys, const uint64_t* keys, const uint32_t* vals,
                       const float* splats, const ws_camera* cam, const ws_config* cfg, uint32_t* ranges,
                       float* image, float* t_final, uint32_t* n_contrib, void* stream) {
    if (!valid_camera(cam) || !valid_config(cfg)) return WS_ERR_INVALID_ARG;
    const void* ptrs[] = {num_keys, keys, vals, splats, ranges, image, t_final, n_contrib};
    for (const void* p : ptrs)
        if (!p || !aligned16(p)) return WS_ERR_INVALID_ARG;
    const Frame f = make_frame(cam, cfg);
    return cuda_status(ws::launch_rasterize(num_keys, 0, keys, vals, splats, f, ranges,
                                            image, t_final, n_contrib, static_cast<cudaStream_t>(stream)));
}

ws_status ws_render_frame_host(int64_t n, const float* h_means, const float* h_log_scales, const float* h_quats,
                               const float* h_opacity_logits, const float* h_sh, const ws_camera* cam,
                               const ws_config* cfg, const ws_frame_buffers* b, float* h_image, void* stream) {
    if (!b || !h_image || n < 0 || n >= (int64_t(1) << 32) || !valid_camera(cam) || !valid_config(cfg))
        return WS_ERR_INVALID_ARG;
    const void* hp[] = {h_means, h_log_scales, h_quats, h_opacity_logits, h_sh};
    if (n > 0)
        for (const void* p : hp)
            if (!p) return WS_ERR_INVALID_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (n > 0) {
        const size_t nn = (size_t)n * sizeof(float);
        const struct { void* dst; const void* src; size_t bytes; } up[] = {
            {b->means, h_means, 3 * nn}, {b->log_scales, h_log_scales, 3 * nn}, {b->quats, h_quats, 4 * nn},
            {b->opacity_logits, h_opacity_logits, nn}, {b->sh, h_sh, 48 * nn}};
        for (const auto& c : up) {
            if (!c.dst) return WS_ERR_INVALID_ARG;
            if (cudaMemcpyAsync(c.dst, c.src, c.bytes, cudaMemcpyHostToDevice, s) != cudaSuccess) return WS_ERR_CUDA;
        }
    }
    ws_status st = ws_preprocess(n, b->means, b->log_scales, b->quats, b->opacity_logits, b->sh, cam, cfg,
                                 b->splats, b->depth, b->rect, b->tiles_touched, stream);
    if (st != WS_OK) return st;
    const int64_t tiles = (int64_t)((cam->width + cfg->tile - 1) / cfg->tile) * ((cam->height + cfg->tile - 1) / cfg->tile);
    int end_bit = 31;
    while ((int64_t(1) << (end_bit - 31)) < tiles) ++end_bit;
    if (end_bit == 31) end_bit = 32;
    // ws_cull then the sort (ws_cull_sort_tiles gives the same results and,
    // on GB300, no gain over the two calls)
    st = ws_cull(n, b->tiles_touched, b->rect, b->depth, cam, cfg, b->offsets, b->keys, b->vals, b->key_capacity,
                 b->num_keys, b->workspace, stream);
    if (st != WS_OK) return st;
    ws_config rc = *cfg;
    int32_t in_alt = 0;
    st = WS_ERR_UNSUPPORTED;
    if (cfg->flags & WS_CFG_SORT_SEGMENTED) {
        st = ws_sort_tiles(b->num_keys, b->key_capacity, end_bit, b->keys, b->vals, b->keys_alt, b->vals_alt, cfg,
                           b->workspace, b->ranges, tiles, &in_alt, stream);
        if (st == WS_OK) rc.flags |= WS_CFG_RANGES_GIVEN;
    }
    if (st == WS_ERR_UNSUPPORTED)
        st = ws_sort(b->num_keys, b->key_capacity, 0, end_bit, b->keys, b->vals, b->keys_alt, b->vals_alt, cfg,
                     b->workspace, &in_alt, stream);
    if (st != WS_OK) return st;
    st = ws_rasterize(b->num_keys, in_alt ? b->keys_alt : b->keys, in_alt ? b->vals_alt : b->vals, b->splats, cam,
                      &rc, b->ranges, b->image, b->t_final, b->n_contrib, stream);
    if (st != WS_OK) return st;
    const size_t img = (size_t)cam->width * cam->height * 3 * sizeof(float);
    return cuda_status(cudaMemcpyAsync(h_image, b->image, img, cudaMemcpyDeviceToHost, s));
}

ws_status ws_preprocess_packed(int64_t n, const float* means, const float* log_scales, const float* quats,
                               const float* opacity_logits, const float* sh, const ws_camera* cam,
                               const ws_config* cfg, float* mean2d, uint32_t* axes, uint32_t* rgba, float* depth,
                               uint16_t* rect, uint32_t* tiles_touched, void* stream) {
    if (n < 0 || n >= (int64_t(1) << 32) || !valid_camera(cam) || !valid_config(cfg)) return WS_ERR_INVALID_ARG;
    if (n == 0) return WS_OK;
    const void* ptrs[] = {means, log_scales, quats, opacity_logits, sh, mean2d, axes, rgba, depth, rect,
                          tiles_touched};
    for (const void* p : ptrs)
        if (!p || !aligned16(p)) return WS_ERR_INVALID_ARG;
    const Frame f = make_frame(cam, cfg);
    if (f.TX > 65535 || f.TY > 65535) return WS_ERR_UNSUPPORTED;
    return cuda_status(ws::launch_preprocess_packed(n, means, log_scales, quats, opacity_logits, sh, f, mean2d, axes,
                                                    rgba, depth, rect, tiles_touched,
                                                    static_cast<cudaStream_t>(stream)));
}

ws_status ws_rasterize_packed(const uint32_t* num_keys, const uint64_t* keys, const uint32_t* vals,
                              const float* mean2d, const uint32_t* axes, const uint32_t* rgba, const ws_camera* cam,
                              const ws_config* cfg, uint32_t* ranges, float* image, float* t_final,
                              uint32_t* n_contrib, void* stream) {
    if (!valid_camera(cam) || !valid_config(cfg)) return WS_ERR_INVALID_ARG;
    const void* ptrs[] = {num_keys, keys, vals, mean2d, axes, rgba, ranges, image, t_final, n_contrib};
    for (const void* p : ptrs)
        if (!p || !aligned16(p)) return WS_ERR_INVALID_ARG;
    const Frame f = make_frame(cam, cfg);
    return cuda_status(ws::launch_rasterize_packed(num_keys, keys, vals, mean2d, axes, rgba, f, ranges, image,
                                                   t_final, n_contrib, static_cast<cudaStream_t>(stream)));
}

size_t ws_quads_workspace_bytes(int64_t n, int64_t key_capacity, const ws_camera* cam, const ws_config* cfg) {
    if (n < 0 || n >= (int64_t(1) << 31) || key_capacity < 0 || key_capacity >= (int64_t(1) << 31)) return 0;
    if (!valid_camera(cam) || !valid_config(cfg)) return 0;
    const Frame f = make_frame(cam, cfg);
    return ws::quad_layout(n, key_capacity, (int64_t)f.TX * f.TY).total;
}

ws_status ws_render_quads(int64_t n, const float* splats, const float* depth, const uint32_t* tiles_touched,
                          const ws_camera* cam,
                          const ws_config* cfg, int64_t key_capacity, uint64_t* keys, uint32_t* vals,
                          uint64_t* keys_alt, uint32_t* vals_alt, uint32_t* num_keys, float* image, float* t_final,
                          void* workspace, void* stream) {
    if (n < 0 || n >= (int64_t(1) << 31) || key_capacity < 0 || key_capacity >= (int64_t(1) << 31))
        return WS_ERR_INVALID_ARG;
    if (!valid_camera(cam) || !valid_config(cfg)) return WS_ERR_INVALID_ARG;
    const void* ptrs[] = {num_keys, image, t_final, workspace};
    for (const void* p : ptrs)
        if (!p || !aligned16(p)) return WS_ERR_INVALID_ARG;
    if (n > 0) {
        const void* in[] = {splats, depth, tiles_touched};
        for (const void* p : in)
            if (!p || !aligned16(p)) return WS_ERR_INVALID_ARG;
    }
    if (key_capacity > 0) {
        const void* kp[] = {keys, vals, keys_alt, vals_alt};
        for (const void* p : kp)
            if (!p || !aligned16(p)) return WS_ERR_INVALID_ARG;
    }
    const Frame f = make_frame(cam, cfg);
    if (f.TX > 65535 || f.TY > 65535) return WS_ERR_UNSUPPORTED;
    return cuda_status(ws::launch_render_quads(n, splats, depth, tiles_touched, f, key_capacity,
                                               keys, vals, keys_alt, vals_alt, num_keys, image, t_final, workspace,
                                               static_cast<cudaStream_t>(stream)));
}

ws_status ws_rasterize_backward(int64_t n, const float* means, const float* log_scales,
                                const float* quats, const float* opacity_logits, const float* sh,
                                const ws_camera* cam, const ws_config* cfg, const float* splats,
                                const uint16_t* rect, const uint32_t* offsets,
                                const uint32_t* tiles_touched, const uint32_t* vals,
                                const uint32_t* ranges, const float* t_final, const uint32_t* n_contrib,
                                const float* d_image, int64_t key_capacity, float* d_means,
                                float* d_log_scales, float* d_quats, float* d_opacity_logits,
                                float* d_sh, void* workspace, void* stream) {
    (void)opacity_logits;  // sigma is read back from the splat records
    if (n < 0 || n >= (int64_t(1) << 32) || key_capacity < 0 || key_capacity >= (int64_t(1) << 31))
        return WS_ERR_INVALID_ARG;
    if (!valid_camera(cam) || !valid_config(cfg)) return WS_ERR_INVALID_ARG;
    const void* ptrs[] = {ranges, t_final, n_contrib, d_image, workspace, offsets};
    for (const void* p : ptrs)
        if (!p || !aligned16(p)) return WS_ERR_INVALID_ARG;
    if (n > 0) {
        const void* per[] = {means, log_scales, quats, sh, splats, rect,
                             tiles_touched, d_means, d_log_scales, d_quats, d_opacity_logits, d_sh};
        for (const void* p : per)
            if (!p || !aligned16(p)) return WS_ERR_INVALID_ARG;
    }
    if (key_capacity > 0 && (!vals || !aligned16(vals))) return WS_ERR_INVALID_ARG;
    const Frame f = make_frame(cam, cfg);
    char* ws_base = static_cast<char*>(workspace);
    return cuda_status(ws::launch_backward(n, means, log_scales, quats, sh, f, splats,
                                           rect, offsets, tiles_touched, vals, ranges, t_final, n_contrib,
                                           d_image, d_means, d_log_scales, d_quats, d_opacity_logits, d_sh,
                                           key_capacity, ws_base + layout(0, key_capacity).bwd,
                                           static_cast<cudaStream_t>(stream)));
}

size_t ws_batch_workspace_bytes(int64_t n, int32_t views, const ws_camera* cams, int64_t key_capacity,
                                const ws_config* cfg) {
    ws::FrameTable ft;
    if (n < 0 || key_capacity < 0 || key_capacity >= (int64_t(1) << 31) || !make_table(views, cams, cfg, ft))
        return 0;
    if (!ws::sort_digit_supported(cfg->digit_bits) || n * views >= (int64_t(1) << 32)) return 0;
    return layout(n * views, key_capacity).total;
}

int32_t ws_batch_max_views(void) { return ws::kMaxViews; }

ws_status ws_preprocess_batch(int64_t n, const float* means, const float* log_scales, const float* quats,
                              const float* opacity_logits, const float* sh, int32_t views, const ws_camera* cams,
                              const ws_config* cfg, float* splats, float* depth, uint16_t* rect,
                              uint32_t* tiles_touched, void* stream) {
    ws::FrameTable ft;
    if (n < 0 || !make_table(views, cams, cfg, ft) || n * views >= (int64_t(1) << 32)) return WS_ERR_INVALID_ARG;
    if (n == 0) return WS_OK;
    const void* ptrs[] = {means, log_scales, quats, opacity_logits, sh, splats, depth, rect, tiles_touched};
    for (const void* p : ptrs)
        if (!p || !aligned16(p)) return WS_ERR_INVALID_ARG;
    return cuda_status(ws::launch_preprocess_batch(n, means, log_scales, quats, opacity_logits, sh, ft, splats,
                                                   depth, rect, tiles_touched,
                                                   static_cast<cudaStream_t>(stream)));
}

ws_status ws_cull_batch(int64_t n, int32_t views, const ws_camera* cams, const ws_config* cfg,
                        const uint32_t* tiles_touched, const uint16_t* rect, const float* depth, uint32_t* offsets,
                        uint64_t* keys, uint32_t* vals, int64_t key_capacity, uint32_t* num_keys, void* workspace,
                        void* stream) {
    ws::FrameTable ft;
    if (n < 0 || key_capacity < 0 || key_capacity >= (int64_t(1) << 31) || !make_table(views, cams, cfg, ft) ||
        n * views >= (int64_t(1) << 32) || !ws::sort_digit_supported(cfg->digit_bits))
        return WS_ERR_INVALID_ARG;
    const void* ptrs[] = {offsets, num_keys, workspace};
    for (const void* p : ptrs)
        if (!p || !aligned16(p)) return WS_ERR_INVALID_ARG;
    if (n > 0) {
        const void* in[] = {tiles_touched, rect, depth};
        for (const void* p : in)
            if (!p || !aligned16(p)) return WS_ERR_INVALID_ARG;
    }
    if (key_capacity > 0 && (!keys || !vals || !aligned16(keys) || !aligned16(vals))) return WS_ERR_INVALID_ARG;
    const Layout L = layout(n * views, key_capacity);
    char* ws_base = static_cast<char*>(workspace);
    return cuda_status(ws::launch_cull_batch(n, make_grid(ft), tiles_touched, rect, depth, offsets, keys, vals,
                                             key_capacity, num_keys, reinterpret_cast<uint32_t*>(ws_base + L.status),
                                             ws_base + L.cull, static_cast<cudaStream_t>(stream)));
}

ws_status ws_rasterize_batch(const uint32_t* num_keys, const uint64_t* keys, const uint32_t* vals, int64_t n,
                             const float* splats, int32_t views, const ws_camera* cams, const ws_config* cfg, uint32_t* ranges,
                             float* image, float* t_final, uint32_t* n_contrib, void* stream) {
    ws::FrameTable ft;
    if (n < 0 || !make_table(views, cams, cfg, ft)) return WS_ERR_INVALID_ARG;
    const void* ptrs[] = {num_keys, keys, vals, splats, ranges, image, t_final, n_contrib};
    for (const void* p : ptrs)
        if (!p || !aligned16(p)) return WS_ERR_INVALID_ARG;
    return cuda_status(ws::launch_rasterize_batch(num_keys, keys, vals, n, splats, ft, ranges,
                                                  image, t_final, n_contrib, static_cast<cudaStream_t>(stream)));
}

ws_status ws_rasterize_backward_batch(int64_t n, const float* means, const float* log_scales, const float* quats,
                                      const float* sh, int32_t views, const ws_camera* cams, const ws_config* cfg,
                                      const float* splats, const uint16_t* rect, const uint32_t* offsets,
                                      const uint32_t* tiles_touched, const uint32_t* vals, const uint32_t* ranges,
                                      const float* t_final, const uint32_t* n_contrib, const float* d_image,
                                      int64_t key_capacity, float* d_means, float* d_log_scales, float* d_quats,
                                      float* d_opacity_logits, float* d_sh, void* workspace, void* stream) {
    ws::FrameTable ft;
    if (n < 0 || key_capacity < 0 || key_capacity >= (int64_t(1) << 31) || !make_table(views, cams, cfg, ft))
        return WS_ERR_INVALID_ARG;
    const void* ptrs[] = {ranges, t_final, n_contrib, d_image, workspace, offsets};
    for (const void* p : ptrs)
        if (!p || !aligned16(p)) return WS_ERR_INVALID_ARG;
    if (n > 0) {
        const void* per[] = {means, log_scales, quats, sh, splats, rect,
                             tiles_touched, d_means, d_log_scales, d_quats, d_opacity_logits, d_sh};
        for (const void* p : per)
            if (!p || !aligned16(p)) return WS_ERR_INVALID_ARG;
    }
    if (key_capacity > 0 && (!vals || !aligned16(vals))) return WS_ERR_INVALID_ARG;
    char* ws_base = static_cast<char*>(workspace);
    return cuda_status(ws::launch_backward_batch(n, means, log_scales, quats, sh, ft, splats,
                                                 rect, offsets, tiles_touched, vals, ranges, t_final, n_contrib,
                                                 d_image, d_means, d_log_scales, d_quats, d_opacity_logits, d_sh,
                                                 key_capacity, ws_base + layout(0, key_capacity).bwd,
                                                 static_cast<cudaStream_t>(stream)));
}

ws_status ws_render_train_l2(int64_t n, const float* means, const float* log_scales, const float* quats,
                             const float* sh, const ws_camera* cam, const ws_config* cfg, const uint32_t* num_keys,
                             const uint64_t* keys, const uint32_t* vals, const float* splats, const uint16_t* rect,
                             const uint32_t* offsets, const uint32_t* tiles_touched, const float* target,
                             int64_t key_capacity, uint32_t* ranges, float* image, float* t_final,
                             uint32_t* n_contrib, float* d_means, float* d_log_scales, float* d_quats,
                             float* d_opacity_logits, float* d_sh, void* workspace, void* stream) {
    if (n < 0 || n >= (int64_t(1) << 32) || key_capacity < 0 || key_capacity >= (int64_t(1) << 31))
        return WS_ERR_INVALID_ARG;
    if (!valid_camera(cam) || !valid_config(cfg)) return WS_ERR_INVALID_ARG;
    const void* ptrs[] = {num_keys, keys, vals, offsets, target, ranges, image, t_final, n_contrib, workspace};
    for (const void* p : ptrs)
        if (!p || !aligned16(p)) return WS_ERR_INVALID_ARG;
    if (n > 0) {
        const void* per[] = {means, log_scales, quats, sh, splats, rect, tiles_touched, d_means, d_log_scales,
                             d_quats, d_opacity_logits, d_sh};
        for (const void* p : per)
            if (!p || !aligned16(p)) return WS_ERR_INVALID_ARG;
    }
    const Frame f = make_frame(cam, cfg);
    char* ws_base = static_cast<char*>(workspace);
    return cuda_status(ws::launch_train(n, means, log_scales, quats, sh, f, num_keys, keys, vals, splats, rect,
                                        offsets, tiles_touched, target, ranges, image, t_final, n_contrib, d_means,
                                        d_log_scales, d_quats, d_opacity_logits, d_sh, key_capacity,
                                        ws_base + layout(0, key_capacity).bwd, static_cast<cudaStream_t>(stream)));
}

ws_status ws_render_train_l2_batch(int64_t n, const float* means, const float* log_scales, const float* quats,
                                   const float* sh, int32_t views, const ws_camera* cams, const ws_config* cfg,
                                   const uint32_t* num_keys, const uint64_t* keys, const uint32_t* vals,
                                   const float* splats, const uint16_t* rect, const uint32_t* offsets,
                                   const uint32_t* tiles_touched, const float* target, int64_t key_capacity,
                                   uint32_t* ranges, float* image, float* t_final, uint32_t* n_contrib,
                                   float* d_means, float* d_log_scales, float* d_quats, float* d_opacity_logits,
                                   float* d_sh, void* workspace, void* stream) {
    ws::FrameTable ft;
    if (n < 0 || key_capacity < 0 || key_capacity >= (int64_t(1) << 31) || !make_table(views, cams, cfg, ft) ||
        n * views >= (int64_t(1) << 32))
        return WS_ERR_INVALID_ARG;
    const void* ptrs[] = {num_keys, keys, vals, offsets, target, ranges, image, t_final, n_contrib, workspace};
    for (const void* p : ptrs)
        if (!p || !aligned16(p)) return WS_ERR_INVALID_ARG;
    if (n > 0) {
        const void* per[] = {means, log_scales, quats, sh, splats, rect, tiles_touched, d_means, d_log_scales,
                             d_quats, d_opacity_logits, d_sh};
        for (const void* p : per)
            if (!p || !aligned16(p)) return WS_ERR_INVALID_ARG;
    }
    char* ws_base = static_cast<char*>(workspace);
    return cuda_status(ws::launch_train_batch(n, means, log_scales, quats, sh, ft, num_keys, keys, vals, splats, rect,
                                              offsets, tiles_touched, target, ranges, image, t_final, n_contrib,
                                              d_means, d_log_scales, d_quats, d_opacity_logits, d_sh, key_capacity,
                                              (cfg->flags & WS_CFG_PERSISTENT) != 0u,
                                              ws_base + layout(0, key_capacity).bwd,
                                              static_cast<cudaStream_t>(stream)));
}

ws_status ws_image_residual(int64_t count, const float* image, const float* target, float* d_image, void* stream) {
    if (count < 0) return WS_ERR_INVALID_ARG;
    if (count == 0) return WS_OK;
    const void* ptrs[] = {image, target, d_image};
    for (const void* p : ptrs)
        if (!p || !aligned16(p)) return WS_ERR_INVALID_ARG;
    return cuda_status(ws::launch_residual(count, image, target, d_image, static_cast<cudaStream_t>(stream)));
}

ws_status ws_read_status(void* workspace, uint32_t* flags, int32_t clear, void* stream) {
    if (!workspace || !flags || !aligned16(workspace)) return WS_ERR_INVALID_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    uint32_t words[2] = {0, 0};
    cudaError_t e = cudaMemcpyAsync(words, workspace, sizeof(words), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return WS_ERR_CUDA;
    *flags = (words[0] ? WS_FLAG_CAPACITY : 0u) | (words[1] ? WS_FLAG_TIMEOUT : 0u);
    if (clear) {
        e = cudaMemsetAsync(workspace, 0, ws::kStatusBytes, s);
        if (e != cudaSuccess) return WS_ERR_CUDA;
    }
    return WS_OK;
}

}  // extern "C"
