// Deterministic backward of the render path (the paper renders only; §1
// notes the 3DGS representation is differentiable). No float atomics: every
// (tile, splat) pair owns one 9-float record of partial derivatives at its
// emission slot  offsets[g] + (ty - y0) * w + (tx - x0)  (the slot the
// compaction gave it), each record is written exactly once, and each
// Gaussian sums its contiguous records in slot order. Results are therefore
// bitwise reproducible.
//
// k_blend_bwd: one block per tile, one thread per pixel, back to front from
//   the stored final transmittance and last-contributor count. With
//   B = colour behind splat i normalised by T_{i+1} (B starts as the
//   background and is updated B <- a c + (1 - a) B):
//     dL/dc_i = a_i T_i dL/dC,   dL/da_i = T_i (c_i - B_i) . dL/dC,
//   then, unless the alpha was clamped at 0.99,
//     sigma dL/dsigma = raw dL/da (raw = sigma G, the unclamped alpha),
//     dL/dpower = a dL/da, power = -1/2 d^T Q d,
//   giving d/dmean = Q d, d/dQ_a = -dx^2/2, d/dQ_b = -dx dy, d/dQ_c = -dy^2/2.
//   (The sigma partial is kept multiplied by sigma: dL/dlogit is then that
//   sum times 1 - sigma.)
//   Each half-warp (a 4x4 pixel sub-block) reduces its 16 pixels with a
//   fixed shuffle tree, the block adds its half-warps in order, and the
//   record goes to the pair's slot.
// k_preprocess_bwd: one thread per Gaussian: slot-ordered sum of its
//   records, then the adjoint of conic = Sigma'^{-1}, Sigma' = T Sigma T^T,
//   T = J W (J's guard-band clamp passes no gradient), the projection of
//   the centre, Sigma = M M^T with M = R(q) diag(exp(log_scale)), the
//   quaternion normalisation, sigma = sigmoid(logit) and the SH colour
//   (clamped channels pass no gradient).
#include "ws_blend.cuh"
#include "ws_common.cuh"
#include "ws_kernels.cuh"
#include "ws_project.cuh"

namespace ws {

namespace {

// Backward records of one tile per block, the tiles taken centre-out
// (centre_out_tile): 2.5 % faster than raster order on the 720p step, where
// the longest lists are near the centre.
template <int TS>
__global__ void __launch_bounds__(TS * TS >= 256 ? 256 : TS * TS)
k_blend_bwd(const uint2* __restrict__ ranges, const uint32_t* __restrict__ vals, const float4* __restrict__ splats,
            const uint2* __restrict__ rect, const uint32_t* __restrict__ offsets, const Frame f,
            const float* __restrict__ t_final, const uint32_t* __restrict__ n_contrib,
            const float* __restrict__ d_image, float* __restrict__ partials) {
    pdl_wait();
    const int t = centre_out_tile(f, blockIdx.x);
    blend_bwd_tile<TS>(f, t, ranges[t], vals, splats, rect,
                       [offsets](uint32_t g) { return __ldg(offsets + g); }, t_final, n_contrib, d_image, partials);
}

// One training step's blend of a tile (forward, L2 residual, backward
// records) in one block: train_tile, the tiles taken centre-out.
template <int TS>
__global__ void __launch_bounds__(TileGeom<TS>::THREADS)
k_train(const uint2* __restrict__ ranges, const uint32_t* __restrict__ vals, const float4* __restrict__ splats,
        const uint2* __restrict__ rect, const uint32_t* __restrict__ offsets, const Frame f,
        const float* __restrict__ target, float* __restrict__ image, float* __restrict__ t_final,
        uint32_t* __restrict__ n_contrib, float* __restrict__ partials) {
    __shared__ TrainSmem<TS> sm;
    pdl_wait();
    const int t = centre_out_tile(f, blockIdx.x);
    train_tile<TS>(f, t, ranges[t], vals, splats, rect,
                   [offsets](uint32_t g) { return __ldg(offsets + g); }, target, image, t_final, n_contrib, partials,
                   sm);
}

constexpr int kPbThreads = 128;

__global__ void __launch_bounds__(kPbThreads, 8)
k_preprocess_bwd(int64_t n, const float* __restrict__ means, const float* __restrict__ log_scales,
                 const float4* __restrict__ quats, const float4* __restrict__ sh, const Frame f,
                 const float4* __restrict__ splats, const uint32_t* __restrict__ offsets, const uint32_t* __restrict__ touched,
                 uint32_t cap, const float* __restrict__ partials, float* __restrict__ d_means,
                 float* __restrict__ d_log_scales, float4* __restrict__ d_quats,
                 float* __restrict__ d_logits, float4* __restrict__ d_sh) {
    __shared__ __align__(16) float s_sh[kPbThreads / kWarp][kWarp * kShPad];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t i = (int64_t)blockIdx.x * kPbThreads + threadIdx.x;
    const bool valid = i < n;
    pdl_wait();
    const uint32_t cnt = valid ? __ldg(touched + i) : 0u;
    const bool vis = cnt > 0;

    // The SH records of this warp's visible Gaussians are copied into shared
    // memory asynchronously (16-byte copies, coalesced across the warp) while
    // the pair records are summed and the geometry adjoint runs.
    const int64_t warp_first = (int64_t)blockIdx.x * kPbThreads + warp * kWarp;
    float* stage = s_sh[warp];
    const uint32_t need = __ballot_sync(kFull, vis);
    if (need) {
        const float4* src = sh + warp_first * 12;
#pragma unroll
        for (int r = 0; r < 12; ++r) {
            const int v = lane + r * kWarp;
            const int g = v / 12, c = v - g * 12;
            if ((need >> g) & 1u) cp_async16(stage + g * kShPad + 4 * c, src + v);
        }
        asm volatile("cp.async.commit_group;" ::: "memory");
    }

    float gm[3] = {0.f, 0.f, 0.f}, gls[3] = {0.f, 0.f, 0.f}, gq[4] = {0.f, 0.f, 0.f, 0.f}, glogit = 0.f;
    float pr[kPart];
#pragma unroll
    for (int c = 0; c < kPart; ++c) pr[c] = 0.f;
    float X[3] = {0.f, 0.f, 0.f};
    float col[3] = {0.f, 0.f, 0.f};
    if (vis) {
        const uint32_t first = __ldg(offsets + i);
        // pairs at slots past the key capacity were dropped by the emission
        // (the frame carries WS_FLAG_CAPACITY): their records do not exist
        const uint32_t nrec = first >= cap ? 0u : min(cnt, cap - first);
        X[0] = __ldg(means + 3 * i);
        X[1] = __ldg(means + 3 * i + 1);
        X[2] = __ldg(means + 3 * i + 2);
        const float sig = __ldg(splats + kSplatVec4 * i + 1).w;
        const float4 q4 = __ldg(quats + i);
        const float ls[3] = {__ldg(log_scales + 3 * i), __ldg(log_scales + 3 * i + 1), __ldg(log_scales + 3 * i + 2)};
        const float4 cl = __ldg(splats + kSplatVec4 * i + 2);
        col[0] = cl.x;
        col[1] = cl.y;
        col[2] = cl.z;
        // slot-ordered sum of this Gaussian's pair records
        sum_pair_records(partials + (size_t)first * kPart, nrec, pr);
        glogit = pr[5] * (1.f - sig);  // pr[5] = sigma dL/dsigma
        splat_adjoint(f, X, q4, ls, pr, cl.w, gm, gls, gq);  // cl.w: the axis basis's t
    }

    // SH colour adjoint; gradients staged back through shared memory for
    // coalesced writes (zeros for Gaussians that are not visible).
    const int64_t avail = n - warp_first;
    const int nvec = avail <= 0 ? 0 : (int)(avail >= kWarp ? kWarp * 12 : avail * 12);
    if (need) {
        asm volatile("cp.async.wait_group 0;" ::: "memory");
        __syncwarp();
    }
    float* mine = stage + lane * kShPad;
    if (vis) {
        // the SH gradients overwrite this lane's staged coefficients in place
        // (sh_adjoint reads every coefficient before it writes a gradient)
        sh_adjoint(f, X, mine, col, pr, gm, mine, false);
    } else if (need) {
#pragma unroll
        for (int k = 0; k < 48; ++k) mine[k] = 0.f;
    }
    if (need) {
        __syncwarp();
        float4* dst = d_sh + warp_first * 12;
#pragma unroll
        for (int r = 0; r < 12; ++r) {
            const int v = lane + r * kWarp;
            if (v < nvec) {
                const int g = v / 12, c = v - g * 12;
                dst[v] = *reinterpret_cast<const float4*>(stage + g * kShPad + 4 * c);
            }
        }
    } else {
        // no visible Gaussian in this warp: zero gradients, coalesced
        float4* dst = d_sh + warp_first * 12;
        const float4 zero = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
        for (int r = 0; r < 12; ++r) {
            const int v = lane + r * kWarp;
            if (v < nvec) dst[v] = zero;
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

}  // namespace

size_t backward_scratch_bytes(int64_t key_capacity) {
    return (size_t)(key_capacity > 0 ? key_capacity : 1) * kPart * sizeof(float);
}

cudaError_t launch_backward(int64_t n, const float* means, const float* log_scales, const float* quats,
                            const float* sh, const Frame& f, const float* splats, const uint16_t* rect,
                            const uint32_t* offsets, const uint32_t* tiles_touched,
                            const uint32_t* vals, const uint32_t* ranges, const float* t_final,
                            const uint32_t* n_contrib, const float* d_image, float* d_means,
                            float* d_log_scales, float* d_quats, float* d_logits, float* d_sh,
                            int64_t key_capacity, void* scratch, cudaStream_t stream) {
    float* partials = static_cast<float*>(scratch);
    const int ntiles = f.TX * f.TY;
    const uint2* r2 = reinterpret_cast<const uint2*>(ranges);
    const float4* s4 = reinterpret_cast<const float4*>(splats);
    const uint2* rc = reinterpret_cast<const uint2*>(rect);
    cudaError_t e = cudaSuccess;
    if (ntiles > 0) {
        switch (f.TS) {
            case 8:
                e = launch_pdl(k_blend_bwd<8>, dim3(ntiles), dim3(64), 0, stream, r2, vals, s4, rc, offsets, f,
                               t_final, n_contrib, d_image, partials);
                break;
            case 16:
                e = launch_pdl(k_blend_bwd<16>, dim3(ntiles), dim3(256), 0, stream, r2, vals, s4, rc, offsets, f,
                               t_final, n_contrib, d_image, partials);
                break;
            case 32:
                e = launch_pdl(k_blend_bwd<32>, dim3(ntiles), dim3(256), 0, stream, r2, vals, s4, rc, offsets, f,
                               t_final, n_contrib, d_image, partials);
                break;
            default:
                return cudaErrorInvalidValue;
        }
        if (e != cudaSuccess) return e;
    }
    if (n > 0) {
        const int64_t blocks = (n + kPbThreads - 1) / kPbThreads;
        e = launch_pdl(k_preprocess_bwd, dim3((unsigned)blocks), dim3(kPbThreads), 0, stream, n, means, log_scales,
                       reinterpret_cast<const float4*>(quats), reinterpret_cast<const float4*>(sh), f, s4,
                       offsets, tiles_touched, (uint32_t)key_capacity, (const float*)partials, d_means, d_log_scales,
                       reinterpret_cast<float4*>(d_quats), d_logits, reinterpret_cast<float4*>(d_sh));
    }
    return e;
}

cudaError_t launch_train(int64_t n, const float* means, const float* log_scales, const float* quats, const float* sh,
                         const Frame& f, const uint32_t* num_keys, const uint64_t* keys, const uint32_t* vals,
                         const float* splats, const uint16_t* rect, const uint32_t* offsets,
                         const uint32_t* tiles_touched, const float* target, uint32_t* ranges, float* image,
                         float* t_final, uint32_t* n_contrib, float* d_means, float* d_log_scales, float* d_quats,
                         float* d_logits, float* d_sh, int64_t key_capacity, void* scratch, cudaStream_t stream) {
    float* partials = static_cast<float*>(scratch);
    const int ntiles = f.TX * f.TY;
    const float4* s4 = reinterpret_cast<const float4*>(splats);
    const uint2* rc = reinterpret_cast<const uint2*>(rect);
    cudaError_t e = cudaSuccess;
    if (ntiles > 0) {
        e = launch_tile_ranges(keys, num_keys, ranges, (uint32_t)ntiles, f.flags, stream);
        if (e != cudaSuccess) return e;
        const uint2* r2 = reinterpret_cast<const uint2*>(ranges);
        switch (f.TS) {
            case 8:
                e = launch_pdl(k_train<8>, dim3(ntiles), dim3(TileGeom<8>::THREADS), 0, stream, r2, vals, s4, rc,
                               offsets, f, target, image, t_final, n_contrib, partials);
                break;
            case 16:
                e = launch_pdl(k_train<16>, dim3(ntiles), dim3(TileGeom<16>::THREADS), 0, stream, r2, vals, s4, rc,
                               offsets, f, target, image, t_final, n_contrib, partials);
                break;
            case 32:
                e = launch_pdl(k_train<32>, dim3(ntiles), dim3(TileGeom<32>::THREADS), 0, stream, r2, vals, s4, rc,
                               offsets, f, target, image, t_final, n_contrib, partials);
                break;
            default:
                return cudaErrorInvalidValue;
        }
        if (e != cudaSuccess) return e;
    }
    if (n > 0) {
        const int64_t blocks = (n + kPbThreads - 1) / kPbThreads;
        e = launch_pdl(k_preprocess_bwd, dim3((unsigned)blocks), dim3(kPbThreads), 0, stream, n, means, log_scales,
                       reinterpret_cast<const float4*>(quats), reinterpret_cast<const float4*>(sh), f, s4,
                       offsets, tiles_touched, (uint32_t)key_capacity, (const float*)partials, d_means, d_log_scales,
                       reinterpret_cast<float4*>(d_quats), d_logits, reinterpret_cast<float4*>(d_sh));
    }
    return e;
}

}  // namespace ws
