// Many views of one scene as one batch: the same per-Gaussian projection,
// per-tile blend and adjoint as the single-view path (shared device code, so
// every view's image is bit-identical to rendering it alone), organised so
// the scene is read once for all views.
//
//   k_preprocess_batch   one thread per Gaussian; its inputs (236 B, SH
//                        staged in shared memory) are read once and every
//                        view is projected from registers; outputs are
//                        view-major and written coalesced per view.
//   compaction / sort    the single-view kernels over V*n items, with tile
//                        ids offset into one global tile grid, so one sort
//                        orders every view's (tile, depth) keys.
//   k_blend_batch        one launch over every (view, tile) work item.
//   k_blend_bwd_batch    likewise, records at each pair's emission slot.
//   k_preprocess_bwd_batch  one thread per Gaussian: for each view in order,
//                        the slot-ordered sum of its records and that view's
//                        adjoint, accumulated in view order (deterministic).
#include "ws_blend.cuh"
#include "ws_common.cuh"
#include "ws_kernels.cuh"
#include "ws_project.cuh"

namespace ws {

namespace {

constexpr int kBatchThreads = 128;

__global__ void __launch_bounds__(kBatchThreads)
k_preprocess_batch(int64_t n, const float* __restrict__ means, const float* __restrict__ log_scales,
                   const float4* __restrict__ quats, const float* __restrict__ logits,
                   const float4* __restrict__ sh, const FrameTable ft, float4* __restrict__ splats,
                   float* __restrict__ depth, uint2* __restrict__ rect, uint32_t* __restrict__ tiles_touched) {
    __shared__ __align__(16) float s_sh[kBatchThreads / kWarp][kWarp * kShPad];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t i = (int64_t)blockIdx.x * kBatchThreads + threadIdx.x;
    const bool valid = i < n;
    const int64_t warp_first = (int64_t)blockIdx.x * kBatchThreads + warp * kWarp;
    pdl_wait();

    float logit = 0.f, x = 0.f, y = 0.f, z = 0.f, l0 = 0.f, l1 = 0.f, l2 = 0.f;
    float4 q = make_float4(0.f, 0.f, 0.f, 0.f);
    if (valid) {
        logit = __ldg(logits + i);
        x = __ldg(means + 3 * i);
        y = __ldg(means + 3 * i + 1);
        z = __ldg(means + 3 * i + 2);
        q = __ldg(quats + i);
        l0 = __ldg(log_scales + 3 * i);
        l1 = __ldg(log_scales + 3 * i + 1);
        l2 = __ldg(log_scales + 3 * i + 2);
    }
    const bool opaque_enough = valid && passes_opacity(ft.f[0], logit);
    const uint32_t need = __ballot_sync(kFull, opaque_enough);
    float* stage = s_sh[warp];
    if (need) {
        const float4* src = sh + warp_first * 12;
#pragma unroll
        for (int r = 0; r < 12; ++r) {
            const int v = lane + r * kWarp;
            const int g = v / 12, c = v - g * 12;
            if ((need >> g) & 1u) cp_async16(stage + g * kShPad + 4 * c, src + v);
        }
        asm volatile("cp.async.commit_group;" ::: "memory");
        asm volatile("cp.async.wait_group 0;" ::: "memory");
        __syncwarp();
    }
    for (int v = 0; v < ft.views; ++v) {
        const Frame& f = ft.f[v];
        const int64_t o = (int64_t)v * n + i;
        bool vis = false;
        Projection P;
        if (valid) {
            const float d = view_depth(f, x, y, z);
            depth[o] = d;
            vis = opaque_enough && d > f.znear;
            if (vis) vis = project_splat(f, x, y, z, q, l0, l1, l2, logit, P);
        }
        float3 c3 = make_float3(0.f, 0.f, 0.f);
        if (vis) {
            const float dx = x - f.campos[0], dy = y - f.campos[1], dz = z - f.campos[2];
            const float inv = rsqrtf(dx * dx + dy * dy + dz * dz);
            sh_eval(dx * inv, dy * inv, dz * inv, stage + lane * kShPad, c3);
        }
        // every lane stores its entries (zeros where culled): whole sectors
        if (valid) {
            store_splat(splats + kSplatVec4 * o, vis, P, c3);
            rect[o] = vis ? make_uint2(P.x0 | (P.y0 << 16), P.x1 | (P.y1 << 16)) : make_uint2(0u, 0u);
            tiles_touched[o] = vis ? (P.x1 - P.x0 + 1) * (P.y1 - P.y0 + 1) : 0u;
        }
    }
}

template <int TS>
__global__ void __launch_bounds__(TS * TS, blend_min_blocks<TS>())
k_blend_batch(const uint2* __restrict__ ranges, const uint32_t* __restrict__ vals, int64_t n,
              const float4* __restrict__ splats, const FrameTable ft,
              float* __restrict__ image, float* __restrict__ t_final, uint32_t* __restrict__ n_contrib) {
    pdl_wait();
    const uint32_t t = blockIdx.x;
    const int v = view_of_tile(ft.tile_off, ft.views, t);
    const uint64_t vo = (uint64_t)v * (uint64_t)n, po = ft.pix_off[v];
    const FloatSplats sp{splats + kSplatVec4 * vo};
    blend_tile<TS>(ft.f[v], (int)(t - ft.tile_off[v]), ranges[t], vals, sp, image + 3 * po, t_final + po,
                   n_contrib + po);
}

template <int TS>
__global__ void __launch_bounds__(TS * TS >= 256 ? 256 : TS * TS)
k_blend_bwd_batch(const uint2* __restrict__ ranges, const uint32_t* __restrict__ vals, int64_t n,
                  const float4* __restrict__ splats, const uint2* __restrict__ rect,
                  const uint32_t* __restrict__ offsets, const FrameTable ft, const float* __restrict__ t_final,
                  const uint32_t* __restrict__ n_contrib, const float* __restrict__ d_image,
                  float* __restrict__ partials) {
    pdl_wait();
    const uint32_t t = blockIdx.x;
    const int v = view_of_tile(ft.tile_off, ft.views, t);
    const uint64_t vo = (uint64_t)v * (uint64_t)n, po = ft.pix_off[v];
    const uint32_t* voff = offsets + vo;
    blend_bwd_tile<TS>(ft.f[v], (int)(t - ft.tile_off[v]), ranges[t], vals, splats + kSplatVec4 * vo, rect + vo, [voff](uint32_t g) { return __ldg(voff + g); }, t_final + po,
                       n_contrib + po, d_image + 3 * po, partials);
}

// One training step's blend over every (view, tile) item: train_tile per
// item. PERSISTENT = false: one block per item. PERSISTENT = true: a grid of
// as many blocks as fit on the GPU at once, block b taking items b, b + G,
// b + 2G, ... (G = the grid size) in that fixed order, so the assignment is
// static and neighbouring blocks work on neighbouring tiles; no block waits
// on another.
template <int TS, bool PERSISTENT>
__global__ void __launch_bounds__(TileGeom<TS>::THREADS)
k_train_batch(const uint2* __restrict__ ranges, const uint32_t* __restrict__ vals, int64_t n,
              const float4* __restrict__ splats, const uint2* __restrict__ rect,
              const uint32_t* __restrict__ offsets, const FrameTable ft, const float* __restrict__ target,
              float* __restrict__ image, float* __restrict__ t_final, uint32_t* __restrict__ n_contrib,
              float* __restrict__ partials) {
    __shared__ TrainSmem<TS> sm;
    pdl_wait();
    const uint32_t ntiles = ft.tile_off[ft.views];
    const uint32_t stride = PERSISTENT ? gridDim.x : ntiles;
    for (uint32_t t = blockIdx.x; t < ntiles; t += stride) {
        const int v = view_of_tile(ft.tile_off, ft.views, t);
        const uint64_t vo = (uint64_t)v * (uint64_t)n, po = ft.pix_off[v];
        const uint32_t* voff = offsets + vo;
        train_tile<TS>(ft.f[v], (int)(t - ft.tile_off[v]), ranges[t], vals, splats + kSplatVec4 * vo, rect + vo,
                       [voff](uint32_t g) { return __ldg(voff + g); }, target + 3 * po, image + 3 * po,
                       t_final + po, n_contrib + po, partials, sm);
    }
}

__global__ void __launch_bounds__(kBatchThreads)
k_preprocess_bwd_batch(int64_t n, const float* __restrict__ means, const float* __restrict__ log_scales,
                       const float4* __restrict__ quats, const float4* __restrict__ sh, const FrameTable ft,
                       const float4* __restrict__ splats, const uint32_t* __restrict__ offsets,
                       const uint32_t* __restrict__ touched,
                       uint32_t cap, const float* __restrict__ partials, float* __restrict__ d_means,
                       float* __restrict__ d_log_scales, float4* __restrict__ d_quats,
                       float* __restrict__ d_logits, float4* __restrict__ d_sh) {
    __shared__ __align__(16) float s_sh[kBatchThreads / kWarp][kWarp * kShPad];
    __shared__ __align__(16) float s_gsh[kBatchThreads / kWarp][kWarp * kShPad];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t i = (int64_t)blockIdx.x * kBatchThreads + threadIdx.x;
    const bool valid = i < n;
    const int64_t warp_first = (int64_t)blockIdx.x * kBatchThreads + warp * kWarp;
    const int64_t avail = n - warp_first;
    const int nvec = avail <= 0 ? 0 : (int)(avail >= kWarp ? kWarp * 12 : avail * 12);
    pdl_wait();

    float X[3] = {0.f, 0.f, 0.f}, ls[3] = {0.f, 0.f, 0.f};
    float4 q4 = make_float4(0.f, 0.f, 0.f, 0.f);
    if (valid) {
        X[0] = __ldg(means + 3 * i);
        X[1] = __ldg(means + 3 * i + 1);
        X[2] = __ldg(means + 3 * i + 2);
        ls[0] = __ldg(log_scales + 3 * i);
        ls[1] = __ldg(log_scales + 3 * i + 1);
        ls[2] = __ldg(log_scales + 3 * i + 2);
        q4 = __ldg(quats + i);
    }
    // stage this warp's SH coefficients; zero the SH gradient accumulators
    float* stage = s_sh[warp];
    float* gsh = s_gsh[warp] + lane * kShPad;
    {
        const float4* src = sh + warp_first * 12;
#pragma unroll
        for (int r = 0; r < 12; ++r) {
            const int v = lane + r * kWarp;
            if (v < nvec) {
                const int g = v / 12, c = v - g * 12;
                *reinterpret_cast<float4*>(stage + g * kShPad + 4 * c) = __ldg(src + v);
            }
        }
#pragma unroll
        for (int k = 0; k < 48; ++k) gsh[k] = 0.f;
        __syncwarp();
    }
    float gm[3] = {0.f, 0.f, 0.f}, gls[3] = {0.f, 0.f, 0.f}, gq[4] = {0.f, 0.f, 0.f, 0.f}, glogit = 0.f;
    // The next view's pair count and first slot are loaded one view ahead, so
    // their latency overlaps this view's adjoint.
    uint32_t cnt_next = valid ? __ldg(touched + i) : 0u;
    uint32_t off_next = valid ? __ldg(offsets + i) : 0u;
    for (int v = 0; v < ft.views; ++v) {
        const int64_t o = (int64_t)v * n + i;
        const uint32_t cnt = cnt_next, first = off_next;
        if (valid && v + 1 < ft.views) {
            cnt_next = __ldg(touched + o + n);
            off_next = __ldg(offsets + o + n);
        }
        if (cnt == 0) continue;
        float pr[kPart];
#pragma unroll
        for (int c = 0; c < kPart; ++c) pr[c] = 0.f;
        // records past the key capacity were never written (the emission
        // dropped those pairs and raised WS_FLAG_CAPACITY)
        const uint32_t nrec = first >= cap ? 0u : min(cnt, cap - first);
        sum_pair_records(partials + (size_t)first * kPart, nrec, pr);
        const float sig = __ldg(splats + kSplatVec4 * o + 1).w;  // sigma (the same in every view)
        glogit += pr[5] * (1.f - sig);  // pr[5] = sigma dL/dsigma
        const Frame& f = ft.f[v];
        const float4 cl = __ldg(splats + kSplatVec4 * o + 2);  // colour and the axis basis's t
        splat_adjoint(f, X, q4, ls, pr, cl.w, gm, gls, gq);
        const float col[3] = {cl.x, cl.y, cl.z};
        sh_adjoint(f, X, stage + lane * kShPad, col, pr, gm, gsh, true);
    }
    __syncwarp();
    float4* dst = d_sh + warp_first * 12;
    const float* gstage = s_gsh[warp];
#pragma unroll
    for (int r = 0; r < 12; ++r) {
        const int v = lane + r * kWarp;
        if (v < nvec) {
            const int g = v / 12, c = v - g * 12;
            dst[v] = *reinterpret_cast<const float4*>(gstage + g * kShPad + 4 * c);
        }
    }
    if (valid) {
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            d_means[3 * i + a] = gm[a];
            d_log_scales[3 * i + a] = gls[a];
        }
        d_quats[i] = make_float4(gq[0], gq[1], gq[2], gq[3]);
        d_logits[i] = glogit;
    }
}

__global__ void k_residual(int64_t count, const float4* __restrict__ image, const float4* __restrict__ target,
                           float4* __restrict__ d_image, int64_t count4) {
    pdl_wait();
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < count4; j += (int64_t)gridDim.x * blockDim.x) {
        const float4 a = __ldg(image + j), b = __ldg(target + j);
        d_image[j] = make_float4(a.x - b.x, a.y - b.y, a.z - b.z, a.w - b.w);
    }
    // tail (count not a multiple of 4)
    if (blockIdx.x == 0 && threadIdx.x < (count & 3)) {
        const int64_t k = count4 * 4 + threadIdx.x;
        reinterpret_cast<float*>(d_image)[k] =
            reinterpret_cast<const float*>(image)[k] - reinterpret_cast<const float*>(target)[k];
    }
}

}  // namespace

cudaError_t launch_preprocess_batch(int64_t n, const float* means, const float* log_scales, const float* quats,
                                    const float* logits, const float* sh, const FrameTable& ft, float* splats,
                                    float* depth, uint16_t* rect, uint32_t* tiles_touched, cudaStream_t stream) {
    if (n == 0) return cudaSuccess;
    const int64_t blocks = (n + kBatchThreads - 1) / kBatchThreads;
    return launch_pdl(k_preprocess_batch, dim3((unsigned)blocks), dim3(kBatchThreads), 0, stream, n, means,
                      log_scales, reinterpret_cast<const float4*>(quats), logits, reinterpret_cast<const float4*>(sh),
                      ft, reinterpret_cast<float4*>(splats), depth, reinterpret_cast<uint2*>(rect), tiles_touched);
}

cudaError_t launch_rasterize_batch(const uint32_t* num_keys, const uint64_t* keys, const uint32_t* vals, int64_t n,
                                   const float* splats, const FrameTable& ft, uint32_t* ranges, float* image, float* t_final,
                                   uint32_t* n_contrib, cudaStream_t stream) {
    const uint32_t ntiles = ft.tile_off[ft.views];
    if (ntiles == 0) return cudaSuccess;
    cudaError_t e = launch_tile_ranges(keys, num_keys, ranges, ntiles, ft.f[0].flags, stream);
    if (e != cudaSuccess) return e;
    const uint2* r2 = reinterpret_cast<const uint2*>(ranges);
    const float4* s4 = reinterpret_cast<const float4*>(splats);
    switch (ft.f[0].TS) {
        case 8:
            return launch_pdl(k_blend_batch<8>, dim3(ntiles), dim3(64), 0, stream, r2, vals, n, s4, ft, image,
                              t_final, n_contrib);
        case 16:
            return launch_pdl(k_blend_batch<16>, dim3(ntiles), dim3(256), 0, stream, r2, vals, n, s4, ft, image,
                              t_final, n_contrib);
        case 32:
            return launch_pdl(k_blend_batch<32>, dim3(ntiles), dim3(1024), 0, stream, r2, vals, n, s4, ft, image,
                              t_final, n_contrib);
        default:
            return cudaErrorInvalidValue;
    }
}

cudaError_t launch_backward_batch(int64_t n, const float* means, const float* log_scales, const float* quats,
                                  const float* sh, const FrameTable& ft, const float* splats, const uint16_t* rect,
                                  const uint32_t* offsets, const uint32_t* tiles_touched, const uint32_t* vals,
                                  const uint32_t* ranges, const float* t_final, const uint32_t* n_contrib,
                                  const float* d_image, float* d_means, float* d_log_scales, float* d_quats,
                                  float* d_logits, float* d_sh, int64_t key_capacity, void* scratch,
                                  cudaStream_t stream) {
    float* partials = static_cast<float*>(scratch);
    const uint32_t ntiles = ft.tile_off[ft.views];
    const uint2* r2 = reinterpret_cast<const uint2*>(ranges);
    const float4* s4 = reinterpret_cast<const float4*>(splats);
    const uint2* rc = reinterpret_cast<const uint2*>(rect);
    cudaError_t e = cudaSuccess;
    if (ntiles > 0) {
        switch (ft.f[0].TS) {
            case 8:
                e = launch_pdl(k_blend_bwd_batch<8>, dim3(ntiles), dim3(64), 0, stream, r2, vals, n, s4, rc, offsets,
                               ft, t_final, n_contrib, d_image, partials);
                break;
            case 16:
                e = launch_pdl(k_blend_bwd_batch<16>, dim3(ntiles), dim3(256), 0, stream, r2, vals, n, s4, rc,
                               offsets, ft, t_final, n_contrib, d_image, partials);
                break;
            case 32:
                e = launch_pdl(k_blend_bwd_batch<32>, dim3(ntiles), dim3(256), 0, stream, r2, vals, n, s4, rc,
                               offsets, ft, t_final, n_contrib, d_image, partials);
                break;
            default:
                return cudaErrorInvalidValue;
        }
        if (e != cudaSuccess) return e;
    }
    if (n > 0) {
        const int64_t blocks = (n + kBatchThreads - 1) / kBatchThreads;
        e = launch_pdl(k_preprocess_bwd_batch, dim3((unsigned)blocks), dim3(kBatchThreads), 0, stream, n, means,
                       log_scales, reinterpret_cast<const float4*>(quats), reinterpret_cast<const float4*>(sh), ft, s4,
                       offsets, tiles_touched, (uint32_t)key_capacity, (const float*)partials, d_means,
                       d_log_scales,
                       reinterpret_cast<float4*>(d_quats), d_logits, reinterpret_cast<float4*>(d_sh));
    }
    return e;
}

cudaError_t launch_residual(int64_t count, const float* image, const float* target, float* d_image,
                            cudaStream_t stream) {
    if (count == 0) return cudaSuccess;
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return launch_pdl(k_residual, dim3(sms * 4), dim3(256), 0, stream, count,
                      reinterpret_cast<const float4*>(image), reinterpret_cast<const float4*>(target),
                      reinterpret_cast<float4*>(d_image), count / 4);
}

template <int TS>
cudaError_t launch_train_batch_ts(const uint2* r2, const uint32_t* vals, int64_t n, const float4* s4, const uint2* rc,
                                  const uint32_t* offsets, const FrameTable& ft, const float* target, float* image,
                                  float* t_final, uint32_t* n_contrib, float* partials, bool persistent,
                                  cudaStream_t stream) {
    const uint32_t ntiles = ft.tile_off[ft.views];
    constexpr int kThreads = TileGeom<TS>::THREADS;
    if (!persistent)
        return launch_pdl(k_train_batch<TS, false>, dim3(ntiles), dim3(kThreads), 0, stream, r2, vals, n, s4, rc,
                          offsets, ft, target, image, t_final, n_contrib, partials);
    int dev = 0, sms = 148, occ = 1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_train_batch<TS, true>, kThreads, 0);
    if (e != cudaSuccess) return e;
    const uint32_t grid = min(ntiles, (uint32_t)(sms * (occ > 0 ? occ : 1)));
    return launch_pdl(k_train_batch<TS, true>, dim3(grid), dim3(kThreads), 0, stream, r2, vals, n, s4, rc, offsets,
                      ft, target, image, t_final, n_contrib, partials);
}

cudaError_t launch_train_batch(int64_t n, const float* means, const float* log_scales, const float* quats,
                               const float* sh, const FrameTable& ft, const uint32_t* num_keys, const uint64_t* keys,
                               const uint32_t* vals, const float* splats, const uint16_t* rect,
                               const uint32_t* offsets, const uint32_t* tiles_touched, const float* target,
                               uint32_t* ranges, float* image, float* t_final, uint32_t* n_contrib, float* d_means,
                               float* d_log_scales, float* d_quats, float* d_logits, float* d_sh,
                               int64_t key_capacity, bool persistent, void* scratch, cudaStream_t stream) {
    float* partials = static_cast<float*>(scratch);
    const uint32_t ntiles = ft.tile_off[ft.views];
    const float4* s4 = reinterpret_cast<const float4*>(splats);
    const uint2* rc = reinterpret_cast<const uint2*>(rect);
    cudaError_t e = cudaSuccess;
    if (ntiles > 0) {
        e = launch_tile_ranges(keys, num_keys, ranges, ntiles, ft.f[0].flags, stream);
        if (e != cudaSuccess) return e;
        const uint2* r2 = reinterpret_cast<const uint2*>(ranges);
        switch (ft.f[0].TS) {
            case 8:
                e = launch_train_batch_ts<8>(r2, vals, n, s4, rc, offsets, ft, target, image, t_final, n_contrib,
                                             partials, persistent, stream);
                break;
            case 16:
                e = launch_train_batch_ts<16>(r2, vals, n, s4, rc, offsets, ft, target, image, t_final, n_contrib,
                                              partials, persistent, stream);
                break;
            case 32:
                e = launch_train_batch_ts<32>(r2, vals, n, s4, rc, offsets, ft, target, image, t_final, n_contrib,
                                              partials, persistent, stream);
                break;
            default:
                return cudaErrorInvalidValue;
        }
        if (e != cudaSuccess) return e;
    }
    if (n > 0) {
        const int64_t blocks = (n + kBatchThreads - 1) / kBatchThreads;
        e = launch_pdl(k_preprocess_bwd_batch, dim3((unsigned)blocks), dim3(kBatchThreads), 0, stream, n, means,
                       log_scales, reinterpret_cast<const float4*>(quats), reinterpret_cast<const float4*>(sh), ft, s4,
                       offsets, tiles_touched, (uint32_t)key_capacity, (const float*)partials, d_means,
                       d_log_scales, reinterpret_cast<float4*>(d_quats), d_logits, reinterpret_cast<float4*>(d_sh));
    }
    return e;
}

}  // namespace ws
