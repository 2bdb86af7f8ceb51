// Packed-record variant of the frame (§3.2): the pre-processing stores each
// visible splat's colour and opacity as one RGBA8 word and its ellipse as
// two words of binary16 axes, with a float32 centre: 20 bytes per splat for
// the blend instead of 44. The ellipse axes are v1 = sqrt(l1) e1 and
// v2 = sqrt(l2) e2 of Sigma' = v1 v1^T + v2 v2^T, so the blend rebuilds
// Sigma' from the four halves and inverts it; det Sigma' = (v1 x v2)^2 has no
// cancellation. Everything after the packing (the opacity-aware extent, the
// viewport test, the tile rectangle, the blend) uses the packed values, so
// the rest of the frame is the float path's, on a quantised splat.
//
// Colours are clamped to [0, 1] by the 8-bit encoding (the float path has
// no upper clamp); opacity and colour are within half a step (1/510) of the
// float values, the axes within binary16 rounding (2^-11 relative).
#include <cuda_fp16.h>

#include "ws_blend.cuh"
#include "ws_common.cuh"
#include "ws_kernels.cuh"
#include "ws_project.cuh"

namespace ws {

namespace {

constexpr int kPreThreads = 128;

// x in [0, 1] on 8 bits, to nearest (ties to even).
__device__ __forceinline__ uint32_t quant8(float x) {
    return (uint32_t)rintf(fminf(1.f, fmaxf(0.f, x)) * 255.f);
}

__device__ __forceinline__ uint32_t pack_half2(float a, float b) {
    return (uint32_t)__half_as_ushort(__float2half_rn(a)) |
           ((uint32_t)__half_as_ushort(__float2half_rn(b)) << 16);
}

__device__ __forceinline__ float2 unpack_half2(uint32_t w) {
    return make_float2(__half2float(__ushort_as_half((unsigned short)(w & 0xffffu))),
                       __half2float(__ushort_as_half((unsigned short)(w >> 16))));
}

// Major / minor axes of [[sxx, sxy], [sxy, syy]] with determinant det:
// v1 = sqrt(l1) e1, v2 = sqrt(l2) e2 with e2 = e1 turned by +90 degrees. e1
// comes from whichever row of (Sigma' - l1 I) is better conditioned;
// l2 = det / l1.
__device__ __forceinline__ void ellipse_axes(float sxx, float sxy, float syy, float det, float& v1x, float& v1y,
                                             float& v2x, float& v2y) {
    const float m = 0.5f * (sxx + syy), h = 0.5f * (sxx - syy);
    const float d = sqrtf(fmaf(h, h, sxy * sxy));
    const float l1 = m + d;
    const float l2 = det / l1;
    float ex = 1.f, ey = 0.f;
    if (d > 0.f) {
        if (h >= 0.f) {
            const float nn = hypotf(d + h, sxy);
            ex = (d + h) / nn;
            ey = sxy / nn;
        } else {
            const float nn = hypotf(sxy, d - h);
            ex = sxy / nn;
            ey = (d - h) / nn;
        }
    }
    const float r1 = sqrtf(l1), r2 = sqrtf(fmaxf(l2, 0.f));
    v1x = r1 * ex;
    v1y = r1 * ey;
    v2x = -r2 * ey;
    v2y = r2 * ex;
}

// Sigma' = v1 v1^T + v2 v2^T from the two packed axes, and its determinant
// (v1 x v2)^2. The pre-processing and the blend both rebuild it here.
__device__ __forceinline__ void axes_cov(uint2 w, float& sxx, float& sxy, float& syy, float& det) {
    const float2 v1 = unpack_half2(w.x), v2 = unpack_half2(w.y);
    sxx = fmaf(v1.x, v1.x, v2.x * v2.x);
    sxy = fmaf(v1.x, v1.y, v2.x * v2.y);
    syy = fmaf(v1.y, v1.y, v2.y * v2.y);
    const float cross = fmaf(v1.x, v2.y, -v1.y * v2.x);
    det = cross * cross;
}

// Blend inputs from the packed record.
struct PackedSplats {
    const float2* __restrict__ mean2d;
    const uint2* __restrict__ axes;
    const uint32_t* __restrict__ rgba;
    __device__ __forceinline__ void load(uint32_t g, float ox, float oy, float& x, float& y, float& a, float& b,
                                         float& c, float& op, float4& col) const {
        const float2 m = __ldg(mean2d + g);
        x = __fsub_rn(m.x, ox);
        y = __fsub_rn(m.y, oy);
        float sxx, sxy, syy, det;
        axes_cov(__ldg(axes + g), sxx, sxy, syy, det);
        const float id = 1.f / det;
        a = syy * id;
        b = -sxy * id;
        c = sxx * id;
        const uint32_t p = __ldg(rgba + g);
        const float k = 1.f / 255.f;
        col = make_float4((float)(p & 255u) * k, (float)((p >> 8) & 255u) * k, (float)((p >> 16) & 255u) * k, 0.f);
        op = (float)(p >> 24) * k;
    }
};

__global__ void __launch_bounds__(kPreThreads)
k_preprocess_packed(int64_t n, const float* __restrict__ means, const float* __restrict__ log_scales,
                    const float4* __restrict__ quats, const float* __restrict__ logits,
                    const float4* __restrict__ sh, const Frame f, float2* __restrict__ mean2d,
                    uint2* __restrict__ axes, uint32_t* __restrict__ rgba, float* __restrict__ depth,
                    uint2* __restrict__ rect, uint32_t* __restrict__ tiles_touched) {
    __shared__ __align__(16) float s_sh[kPreThreads / kWarp][kWarp * kShPad];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t i = (int64_t)blockIdx.x * kPreThreads + threadIdx.x;
    const bool valid = i < n;
    const int64_t warp_first = (int64_t)blockIdx.x * kPreThreads + warp * kWarp;
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
    const bool opaque_enough = valid && passes_opacity(f, logit);
    const float d = valid ? view_depth(f, x, y, z) : 0.f;
    // SH records of the lanes that will probably be visible are copied early
    // (overlapping the projection), the rest of the visible ones afterwards;
    // the test is the float path's (ws_preprocess.cu).
    const bool likely = opaque_enough && likely_visible(f, x, y, z, d, l0, l1, l2);
    const uint32_t need = __ballot_sync(kFull, likely);
    float* stage = s_sh[warp];
    const float4* src = sh + warp_first * 12;
    if (need) {
#pragma unroll
        for (int r = 0; r < 12; ++r) {
            const int v = lane + r * kWarp;
            const int g = v / 12, c = v - g * 12;
            if ((need >> g) & 1u) cp_async16(stage + g * kShPad + 4 * c, src + v);
        }
        asm volatile("cp.async.commit_group;" ::: "memory");
    }

    bool vis = false;
    Projection P;
    uint2 ax = make_uint2(0u, 0u);
    uint32_t a8 = 0;
    if (valid) {
        depth[i] = d;
        vis = opaque_enough && d > f.znear;
        float sxx, sxy, syy;
        if (vis) vis = project_core(f, x, y, z, q, l0, l1, l2, P, sxx, sxy, syy);
        if (vis) {
            // pack: opacity on 8 bits, ellipse as binary16 axes
            a8 = quant8(1.f / (1.f + expf(-logit)));
            float v1x, v1y, v2x, v2y;
            // det(Sigma') = sxx / conic c, as project_core formed it (no cancellation)
            ellipse_axes(sxx, sxy, syy, sxx / P.cc, v1x, v1y, v2x, v2y);
            ax = make_uint2(pack_half2(v1x, v1y), pack_half2(v2x, v2y));
            // extent, viewport test and tile rectangle of the packed splat
            float qxx, qxy, qyy, det;
            axes_cov(ax, qxx, qxy, qyy, det);
            const float sig = (float)a8 * (1.f / 255.f);
            const float qc =
                (f.flags & WS_CFG_FIXED_RADIUS) ? 2.f * kLn255 : fmaxf(0.f, 2.f * (kLn255 + logf(sig)));
            vis = det > 0.f && splat_rect(f, P.m4.x, 0.f, P.m4.y, 0.f, sqrtf(qc * qxx), sqrtf(qc * qyy), P);
        }
    }

    const uint32_t late = __ballot_sync(kFull, vis && !likely);
    if (late) {
#pragma unroll
        for (int r = 0; r < 12; ++r) {
            const int v = lane + r * kWarp;
            const int g = v / 12, c = v - g * 12;
            if ((late >> g) & 1u) cp_async16(stage + g * kShPad + 4 * c, src + v);
        }
        asm volatile("cp.async.commit_group;" ::: "memory");
    }
    uint32_t packed_rgba = 0u;
    if (need | late) {
        asm volatile("cp.async.wait_group 0;" ::: "memory");
        __syncwarp();
        if (vis) {
            const float dx = x - f.campos[0], dy = y - f.campos[1], dz = z - f.campos[2];
            const float inv = rsqrtf(dx * dx + dy * dy + dz * dz);
            float3 c3;
            sh_eval(dx * inv, dy * inv, dz * inv, stage + lane * kShPad, c3);
            packed_rgba = quant8(c3.x) | (quant8(c3.y) << 8) | (quant8(c3.z) << 16) | (a8 << 24);
        }
    }
    // Every lane stores its entries (zeros for a culled Gaussian): whole
    // sectors, no read of partly written ones from DRAM (as in ws_preprocess).
    if (valid) {
        mean2d[i] = vis ? make_float2(P.m4.x, P.m4.y) : make_float2(0.f, 0.f);
        axes[i] = vis ? ax : make_uint2(0u, 0u);
        rgba[i] = packed_rgba;
        rect[i] = vis ? make_uint2(P.x0 | (P.y0 << 16), P.x1 | (P.y1 << 16)) : make_uint2(0u, 0u);
        tiles_touched[i] = vis ? (P.x1 - P.x0 + 1) * (P.y1 - P.y0 + 1) : 0u;
    }
}

template <int TS>
__global__ void __launch_bounds__(TS * TS, blend_min_blocks<TS>())
k_blend_packed(const uint2* __restrict__ ranges, const uint32_t* __restrict__ vals,
               const float2* __restrict__ mean2d, const uint2* __restrict__ axes,
               const uint32_t* __restrict__ rgba, const Frame f, float* __restrict__ image,
               float* __restrict__ t_final, uint32_t* __restrict__ n_contrib) {
    pdl_wait();
    const PackedSplats sp{mean2d, axes, rgba};
    blend_tile<TS>(f, blockIdx.x, ranges[blockIdx.x], vals, sp, image, t_final, n_contrib);
}

}  // namespace

cudaError_t launch_preprocess_packed(int64_t n, const float* means, const float* log_scales, const float* quats,
                                     const float* logits, const float* sh, const Frame& f, float* mean2d,
                                     uint32_t* axes, uint32_t* rgba, float* depth, uint16_t* rect,
                                     uint32_t* tiles_touched, cudaStream_t stream) {
    if (n == 0) return cudaSuccess;
    const int64_t blocks = (n + kPreThreads - 1) / kPreThreads;
    return launch_pdl(k_preprocess_packed, dim3((unsigned)blocks), dim3(kPreThreads), 0, stream, n, means,
                      log_scales, reinterpret_cast<const float4*>(quats), logits,
                      reinterpret_cast<const float4*>(sh), f, reinterpret_cast<float2*>(mean2d),
                      reinterpret_cast<uint2*>(axes), rgba, depth, reinterpret_cast<uint2*>(rect), tiles_touched);
}

cudaError_t launch_rasterize_packed(const uint32_t* num_keys, const uint64_t* keys, const uint32_t* vals,
                                    const float* mean2d, const uint32_t* axes, const uint32_t* rgba, const Frame& f,
                                    uint32_t* ranges, float* image, float* t_final, uint32_t* n_contrib,
                                    cudaStream_t stream) {
    const int ntiles = f.TX * f.TY;
    if (ntiles == 0) return cudaSuccess;
    cudaError_t e = launch_tile_ranges(keys, num_keys, ranges, (uint32_t)ntiles, f.flags, stream);
    if (e != cudaSuccess) return e;
    const uint2* r2 = reinterpret_cast<const uint2*>(ranges);
    const float2* m2 = reinterpret_cast<const float2*>(mean2d);
    const uint2* a2 = reinterpret_cast<const uint2*>(axes);
    switch (f.TS) {
        case 8:
            return launch_pdl(k_blend_packed<8>, dim3(ntiles), dim3(64), 0, stream, r2, vals, m2, a2, rgba, f, image,
                              t_final, n_contrib);
        case 16:
            return launch_pdl(k_blend_packed<16>, dim3(ntiles), dim3(256), 0, stream, r2, vals, m2, a2, rgba, f,
                              image, t_final, n_contrib);
        case 32:
            return launch_pdl(k_blend_packed<32>, dim3(ntiles), dim3(1024), 0, stream, r2, vals, m2, a2, rgba, f,
                              image, t_final, n_contrib);
        default:
            return cudaErrorInvalidValue;
    }
}

}  // namespace ws
