// Pre-processing stage (paper §3.2 with the covariance/colour model of §2.1
// and the opacity culling and opacity-aware extent of §3.4).
//
// One thread per Gaussian, 128-thread blocks. HBM-bound: 236 B of input per
// visible Gaussian (59 floats), 16 B per opacity-culled one (logit + mean).
// The 192-byte SH record is the bulk of the traffic; each warp stages the
// SH of its 32 Gaussians through shared memory with fully coalesced 16-byte
// loads (a per-thread load of a 192-byte stride would touch 32 cache lines
// per instruction), padded to 52 floats so the per-lane float4 reads are
// bank-conflict free.
#include "ws_common.cuh"
#include "ws_kernels.cuh"

namespace ws {

namespace {

constexpr int kPreThreads = 128;
constexpr int kShPad = 52;  // floats per staged SH record (48 used)

// Real SH basis of degree 3 (Condon-Shortley phase, index l*l + l + m) as
// homogeneous polynomials of the unit direction; constants are
// sqrt((2l+1)/(4 pi) (l-|m|)!/(l+|m|)!) times the polynomial's own factor.
__device__ __forceinline__ void sh_eval(float x, float y, float z, const float4* k, float3& out) {
    const float c0 = 0.28209479177387814f;
    const float c1 = 0.4886025119029199f;
    const float c2a = 1.0925484305920792f, c2b = 0.31539156525252005f, c2c = 0.5462742152960396f;
    const float c3a = 0.5900435899266435f, c3b = 2.890611442640554f, c3c = 0.4570457994644658f;
    const float c3d = 0.3731763325901154f, c3e = 1.445305721320277f;
    float xx = x * x, yy = y * y, zz = z * z;
    float b[16];
    b[0] = c0;
    b[1] = -c1 * y;
    b[2] = c1 * z;
    b[3] = -c1 * x;
    b[4] = c2a * x * y;
    b[5] = -c2a * y * z;
    b[6] = c2b * (2.f * zz - xx - yy);
    b[7] = -c2a * x * z;
    b[8] = c2c * (xx - yy);
    b[9] = -c3a * y * (3.f * xx - yy);
    b[10] = c3b * x * y * z;
    b[11] = -c3c * y * (4.f * zz - xx - yy);
    b[12] = c3d * z * (2.f * zz - 3.f * xx - 3.f * yy);
    b[13] = -c3c * x * (4.f * zz - xx - yy);
    b[14] = c3e * z * (xx - yy);
    b[15] = -c3a * x * (xx - 3.f * yy);
    // k holds 48 floats = coefficient-major [16][3] as 12 float4.
    const float* kf = reinterpret_cast<const float*>(k);
    float r = 0.5f, g = 0.5f, bl = 0.5f;
#pragma unroll
    for (int i = 0; i < 16; ++i) {
        r = fmaf(b[i], kf[3 * i + 0], r);
        g = fmaf(b[i], kf[3 * i + 1], g);
        bl = fmaf(b[i], kf[3 * i + 2], bl);
    }
    out = make_float3(fmaxf(r, 0.f), fmaxf(g, 0.f), fmaxf(bl, 0.f));
}

__global__ void __launch_bounds__(kPreThreads)
k_preprocess(int64_t n, const float* __restrict__ means, const float* __restrict__ log_scales,
             const float4* __restrict__ quats, const float* __restrict__ logits,
             const float4* __restrict__ sh, const Frame f, float4* __restrict__ mean2d,
             float* __restrict__ conic, float* __restrict__ depth, float* __restrict__ rgb,
             float* __restrict__ opacity, uint2* __restrict__ rect,
             uint32_t* __restrict__ tiles_touched) {
    __shared__ __align__(16) float s_sh[kPreThreads / kWarp][kWarp * kShPad];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t i = (int64_t)blockIdx.x * kPreThreads + threadIdx.x;
    const bool valid = i < n;

    bool vis = false;
    float logit = valid ? __ldg(logits + i) : 0.f;
    float x = 0.f, y = 0.f, z = 0.f;
    if (valid) {
        x = __ldg(means + 3 * i);
        y = __ldg(means + 3 * i + 1);
        z = __ldg(means + 3 * i + 2);
        // §3.2: the 32-bit float depth, each operation rounded in a fixed order.
        float d = __fadd_rn(__fadd_rn(__fadd_rn(__fmul_rn(f.R[6], x), __fmul_rn(f.R[7], y)),
                                      __fmul_rn(f.R[8], z)),
                            f.t[2]);
        depth[i] = d;
        bool opaque_enough = (double)logit >= kOpacityLogitMin || (f.flags & WS_CFG_NO_OPACITY_CULL);
        vis = opaque_enough && d > f.znear;
    }
    float4 m4 = make_float4(0.f, 0.f, 0.f, 0.f);
    float ca = 0.f, cb = 0.f, cc = 0.f, sigma = 0.f;
    uint32_t x0 = 0, y0 = 0, x1 = 0, y1 = 0;
    if (vis) {
        float4 q = __ldg(quats + i);
        float qn2 = q.x * q.x + q.y * q.y + q.z * q.z + q.w * q.w;
        if (qn2 == 0.f) vis = false;
        if (vis) {
            float inv = rsqrtf(qn2);
            float w = q.x * inv, qx = q.y * inv, qy = q.z * inv, qz = q.w * inv;
            float R[9] = {1.f - 2.f * (qy * qy + qz * qz), 2.f * (qx * qy - w * qz), 2.f * (qx * qz + w * qy),
                          2.f * (qx * qy + w * qz), 1.f - 2.f * (qx * qx + qz * qz), 2.f * (qy * qz - w * qx),
                          2.f * (qx * qz - w * qy), 2.f * (qy * qz + w * qx), 1.f - 2.f * (qx * qx + qy * qy)};
            float s0 = expf(__ldg(log_scales + 3 * i)), s1 = expf(__ldg(log_scales + 3 * i + 1)),
                  s2 = expf(__ldg(log_scales + 3 * i + 2));
            // M = R S, so Sigma = M M^T (§2.1).
            float M[9] = {R[0] * s0, R[1] * s1, R[2] * s2, R[3] * s0, R[4] * s1,
                          R[5] * s2, R[6] * s0, R[7] * s1, R[8] * s2};
            // Camera-space centre in double-float, then the projected centre.
            DF tx = df_affine3(f.R[0], f.R[1], f.R[2], x, y, z, f.t[0]);
            DF ty = df_affine3(f.R[3], f.R[4], f.R[5], x, y, z, f.t[1]);
            DF tz = df_affine3(f.R[6], f.R[7], f.R[8], x, y, z, f.t[2]);
            DF mx = df_scale_add(f.fx, df_div(tx, tz), f.cx);
            DF my = df_scale_add(f.fy, df_div(ty, tz), f.cy);
            m4 = make_float4(mx.hi, my.hi, mx.lo, my.lo);
            // EWA Jacobian with the guard-band clamp, T = J W.
            float rz = 1.f / tz.hi;
            float rx = fminf(f.limx, fmaxf(-f.limx, tx.hi * rz));
            float ry = fminf(f.limy, fmaxf(-f.limy, ty.hi * rz));
            float j00 = f.fx * rz, j02 = -f.fx * rx * rz, j11 = f.fy * rz, j12 = -f.fy * ry * rz;
            float T0[3] = {j00 * f.R[0] + j02 * f.R[6], j00 * f.R[1] + j02 * f.R[7], j00 * f.R[2] + j02 * f.R[8]};
            float T1[3] = {j11 * f.R[3] + j12 * f.R[6], j11 * f.R[4] + j12 * f.R[7], j11 * f.R[5] + j12 * f.R[8]};
            // V = T M (2x3); Sigma' = T Sigma T^T + dilation I = V V^T + dilation I:
            // sums of squares on the diagonal, no cancellation.
            float V0[3], V1[3];
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                V0[k] = T0[0] * M[k] + T0[1] * M[3 + k] + T0[2] * M[6 + k];
                V1[k] = T1[0] * M[k] + T1[1] * M[3 + k] + T1[2] * M[6 + k];
            }
            float sxx = V0[0] * V0[0] + V0[1] * V0[1] + V0[2] * V0[2] + f.dilation;
            float sxy = V0[0] * V1[0] + V0[1] * V1[1] + V0[2] * V1[2];
            float syy = V1[0] * V1[0] + V1[1] * V1[1] + V1[2] * V1[2] + f.dilation;
            float det = fmaf(sxx, syy, -sxy * sxy);
            if (!(det > 0.f)) vis = false;
            if (vis) {
                float id = 1.f / det;
                ca = syy * id;
                cb = -sxy * id;
                cc = sxx * id;
                // sigma and the opacity-aware extent (§3.4): q_c = 2 ln(255 sigma)
                float en = expf(-logit);
                sigma = 1.f / (1.f + en);
                float qc = fmaxf(0.f, 2.f * (kLn255 - log1pf(en)));
                float ex = sqrtf(qc * sxx), ey = sqrtf(qc * syy);
                float lox = __fadd_rn(__fsub_rn(mx.hi, ex), mx.lo), hix = __fadd_rn(__fadd_rn(mx.hi, ex), mx.lo);
                float loy = __fadd_rn(__fsub_rn(my.hi, ey), my.lo), hiy = __fadd_rn(__fadd_rn(my.hi, ey), my.lo);
                bool on = hix >= 0.f && lox < (float)f.W && hiy >= 0.f && loy < (float)f.H;
                if (!on && !(f.flags & WS_CFG_NO_AABB_CULL)) vis = false;
                if (vis) {
                    float its = 1.f / (float)f.TS;  // exact: TS is a power of two
                    x0 = (uint32_t)fminf((float)(f.TX - 1), fmaxf(0.f, floorf(lox * its)));
                    x1 = (uint32_t)fminf((float)(f.TX - 1), fmaxf(0.f, floorf(hix * its)));
                    y0 = (uint32_t)fminf((float)(f.TY - 1), fmaxf(0.f, floorf(loy * its)));
                    y1 = (uint32_t)fminf((float)(f.TY - 1), fmaxf(0.f, floorf(hiy * its)));
                }
            }
        }
    }

    // SH colour for the visible lanes: warp-cooperative staging of the warp's
    // 32 x 192 B SH records, skipped when no lane of the warp survived.
    const int64_t warp_first = (int64_t)blockIdx.x * kPreThreads + warp * kWarp;
    if (__any_sync(kFull, vis)) {
        float* stage = s_sh[warp];
        const int64_t avail = n - warp_first;
        const int nvec = (int)(avail >= kWarp ? kWarp * 12 : avail * 12);
        const float4* src = sh + warp_first * 12;
#pragma unroll
        for (int r = 0; r < 12; ++r) {
            int v = lane + r * kWarp;
            if (v < nvec) {
                float4 val = __ldg(src + v);
                int g = v / 12, c = v - g * 12;
                *reinterpret_cast<float4*>(stage + g * kShPad + 4 * c) = val;
            }
        }
        __syncwarp();
        if (vis) {
            float dx = x - f.campos[0], dy = y - f.campos[1], dz = z - f.campos[2];
            float inv = rsqrtf(dx * dx + dy * dy + dz * dz);
            float4 k[12];
            const float4* mine = reinterpret_cast<const float4*>(stage + lane * kShPad);
#pragma unroll
            for (int r = 0; r < 12; ++r) k[r] = mine[r];
            float3 c3;
            sh_eval(dx * inv, dy * inv, dz * inv, k, c3);
            mean2d[i] = m4;
            conic[3 * i] = ca;
            conic[3 * i + 1] = cb;
            conic[3 * i + 2] = cc;
            rgb[3 * i] = c3.x;
            rgb[3 * i + 1] = c3.y;
            rgb[3 * i + 2] = c3.z;
            opacity[i] = sigma;
            rect[i] = make_uint2(x0 | (y0 << 16), x1 | (y1 << 16));
        }
    }
    if (valid) tiles_touched[i] = vis ? (x1 - x0 + 1) * (y1 - y0 + 1) : 0u;
}

}  // namespace

cudaError_t launch_preprocess(int64_t n, const float* means, const float* log_scales,
                              const float* quats, const float* logits, const float* sh,
                              const Frame& f, float* mean2d, float* conic, float* depth,
                              float* rgb, float* opacity, uint16_t* rect,
                              uint32_t* tiles_touched, cudaStream_t stream) {
    if (n == 0) return cudaSuccess;
    const int64_t blocks = (n + kPreThreads - 1) / kPreThreads;
    k_preprocess<<<(unsigned)blocks, kPreThreads, 0, stream>>>(
        n, means, log_scales, reinterpret_cast<const float4*>(quats), logits,
        reinterpret_cast<const float4*>(sh), f, reinterpret_cast<float4*>(mean2d), conic, depth,
        rgb, opacity, reinterpret_cast<uint2*>(rect), tiles_touched);
    return cudaGetLastError();
}

}  // namespace ws
