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
//     dL/dsigma = G dL/da, dL/dpower = a dL/da, power = -1/2 d^T Q d,
//   giving d/dmean = Q d, d/dQ_a = -dx^2/2, d/dQ_b = -dx dy, d/dQ_c = -dy^2/2.
//   Each warp reduces its 32 pixels with a fixed shuffle tree, the block
//   adds its warps in warp order, and the record goes to the pair's slot.
// k_preprocess_bwd: one thread per Gaussian: slot-ordered sum of its
//   records, then the adjoint of conic = Sigma'^{-1}, Sigma' = T Sigma T^T,
//   T = J W (J's guard-band clamp passes no gradient), the projection of
//   the centre, Sigma = M M^T with M = R(q) diag(exp(log_scale)), the
//   quaternion normalisation, sigma = sigmoid(logit) and the SH colour
//   (clamped channels pass no gradient).
#include "ws_common.cuh"
#include "ws_kernels.cuh"

namespace ws {

namespace {

constexpr int kBwdBatch = 64;
constexpr int kPart = 9;  // dmean x, y; dconic a, b, c; dsigma; drgb r, g, b

struct BwdRec {
    float4 geo;   // tile-relative centre x, y; premultiplied conic A, B
    float4 geo2;  // premultiplied C, opacity, conic a, conic b
    float4 col;   // r, g, b, conic c
};

template <int TS>
__global__ void __launch_bounds__(TS * TS >= 256 ? 256 : TS * TS)
k_blend_bwd(const uint2* __restrict__ ranges, const uint32_t* __restrict__ vals,
            const float4* __restrict__ mean2d, const float* __restrict__ conic,
            const float* __restrict__ opacity, const float* __restrict__ rgb,
            const uint2* __restrict__ rect, const uint32_t* __restrict__ offsets, const Frame f,
            const float* __restrict__ t_final, const uint32_t* __restrict__ n_contrib,
            const float* __restrict__ d_image, float* __restrict__ partials) {
    constexpr int THREADS = TS * TS >= 256 ? 256 : TS * TS;
    constexpr int WARPS = THREADS / 32;
    constexpr int PPT = TS * TS / THREADS;
    constexpr int BW = 8, BH = 4;
    constexpr int BPR = TS / BW;
    constexpr int BROWS = TS / BH;
    __shared__ BwdRec s_rec[kBwdBatch];
    __shared__ uint32_t s_mask[kBwdBatch];
    __shared__ uint32_t s_slot[kBwdBatch];
    __shared__ float s_part[kBwdBatch][WARPS][kPart];
    __shared__ uint32_t s_max[WARPS];

    const int tile = blockIdx.x;
    const int tx = tile % f.TX, ty = tile / f.TX;
    const float ox = (float)(tx * TS), oy = (float)(ty * TS);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint2 range = ranges[tile];
    const uint32_t len = range.y - range.x;

    float px[PPT], py[PPT], T[PPT], dC[PPT][3], Bc[PPT][3];
    uint32_t last[PPT];
    uint32_t wmask = 0;  // union of this warp's block bits
    uint32_t my_max = 0;
#pragma unroll
    for (int k = 0; k < PPT; ++k) {
        const int b = warp + k * WARPS;
        wmask |= 1u << b;
        const int bx = (b % BPR) * BW, by = (b / BPR) * BH;
        const int lx = bx + (lane & 7), ly = by + (lane >> 3);
        px[k] = (float)lx + 0.5f;
        py[k] = (float)ly + 0.5f;
        const int gx = tx * TS + lx, gy = ty * TS + ly;
        const bool inside = gx < f.W && gy < f.H;
        const size_t pix = inside ? (size_t)gy * f.W + gx : 0;
        T[k] = inside ? t_final[pix] : 1.f;
        last[k] = inside ? n_contrib[pix] : 0u;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            dC[k][c] = inside ? d_image[3 * pix + c] : 0.f;
            Bc[k][c] = f.bg[c];
        }
        my_max = max(my_max, last[k]);
    }
    // Block-wide maximum of the last-contributor counts: positions past it
    // are never composited, their records are zero.
    for (int o = 16; o > 0; o >>= 1) my_max = max(my_max, __shfl_xor_sync(kFull, my_max, o));
    if (lane == 0) s_max[warp] = my_max;
    __syncthreads();
    uint32_t max_last = 0;
#pragma unroll
    for (int w = 0; w < WARPS; ++w) max_last = max(max_last, s_max[w]);

    // Zero records for list positions no pixel composited.
    for (uint32_t j = max_last + threadIdx.x; j < len; j += THREADS) {
        const uint32_t g = __ldg(vals + range.x + j);
        const uint2 r = __ldg(rect + g);
        const uint32_t x0 = r.x & 0xffffu, y0 = r.x >> 16, x1 = r.y & 0xffffu;
        const uint32_t slot = __ldg(offsets + g) + (ty - y0) * (x1 - x0 + 1) + (tx - x0);
        float* dst = partials + (size_t)slot * kPart;
#pragma unroll
        for (int c = 0; c < kPart; ++c) dst[c] = 0.f;
    }

    for (int end = (int)max_last; end > 0; end -= kBwdBatch) {
        const int lo = max(0, end - kBwdBatch);
        const int cnt = end - lo;
        __syncthreads();
        for (int j = threadIdx.x; j < cnt; j += THREADS) {
            const uint32_t g = __ldg(vals + range.x + lo + j);
            const float4 m = __ldg(mean2d + g);
            const float a = __ldg(conic + 3 * g), b = __ldg(conic + 3 * g + 1), c = __ldg(conic + 3 * g + 2);
            const float op = __ldg(opacity + g);
            BwdRec r;
            r.geo.x = __fadd_rn(__fsub_rn(m.x, ox), m.z);
            r.geo.y = __fadd_rn(__fsub_rn(m.y, oy), m.w);
            r.geo.z = -0.5f * kLog2e * a;
            r.geo.w = -kLog2e * b;
            r.geo2 = make_float4(-0.5f * kLog2e * c, op, a, b);
            r.col = make_float4(__ldg(rgb + 3 * g), __ldg(rgb + 3 * g + 1), __ldg(rgb + 3 * g + 2), c);
            s_rec[j] = r;
            const float det = fmaf(a, c, -b * b);
            const float qc = fmaxf(0.f, 2.f * (kLn255 + __logf(op)));
            const float ex = sqrtf(qc * c / det) * 1.0001f + 1e-3f;
            const float ey = sqrtf(qc * a / det) * 1.0001f + 1e-3f;
            const float c0 = fmaxf(0.f, ceilf((r.geo.x - ex - (BW - 0.5f)) * (1.f / BW)));
            const float c1 = fminf((float)(BPR - 1), floorf((r.geo.x + ex - 0.5f) * (1.f / BW)));
            const float r0 = fmaxf(0.f, ceilf((r.geo.y - ey - (BH - 0.5f)) * (1.f / BH)));
            const float r1 = fminf((float)(BROWS - 1), floorf((r.geo.y + ey - 0.5f) * (1.f / BH)));
            uint32_t mask = 0;
            if (c0 <= c1 && r0 <= r1) {
                const int ic0 = (int)c0, ic1 = (int)c1, ir0 = (int)r0, ir1 = (int)r1;
                const uint32_t row = ((2u << ic1) - 1u) & ~((1u << ic0) - 1u);
                for (int rr = ir0; rr <= ir1; ++rr) mask |= row << (rr * BPR);
            }
            s_mask[j] = mask;
            const uint2 rc = __ldg(rect + g);
            const uint32_t x0 = rc.x & 0xffffu, y0 = rc.x >> 16, x1 = rc.y & 0xffffu;
            s_slot[j] = __ldg(offsets + g) + (ty - y0) * (x1 - x0 + 1) + (tx - x0);
        }
        for (int e = threadIdx.x; e < cnt * WARPS * kPart; e += THREADS) (&s_part[0][0][0])[e] = 0.f;
        __syncthreads();

        // Back to front over the batch: chunks of 32 from the top, highest
        // set bit first.
        for (int base = ((cnt - 1) >> 5) << 5; base >= 0; base -= 32) {
            const int jj = base + lane;
            uint32_t bits = __ballot_sync(kFull, jj < cnt && (s_mask[jj] & wmask) != 0u);
            while (bits) {
                const int hb = 31 - __clz(bits);
                bits &= ~(1u << hb);
                const int j = base + hb;
                const uint32_t pos = (uint32_t)(lo + j);
                const BwdRec r = s_rec[j];
                const uint32_t m = s_mask[j];
                float acc[kPart];
#pragma unroll
                for (int c = 0; c < kPart; ++c) acc[c] = 0.f;
                bool any = false;
#pragma unroll
                for (int k = 0; k < PPT; ++k) {
                    if (!((m >> (warp + k * WARPS)) & 1u)) continue;  // warp-uniform
                    if (pos >= last[k]) continue;
                    const float dx = px[k] - r.geo.x, dy = py[k] - r.geo.y;
                    const float G = ex2_approx(splat_power2(dx, dy, r.geo.z, r.geo.w, r.geo2.x));
                    const float raw = __fmul_rn(r.geo2.y, G);
                    const float alpha = fminf(kAlphaMax, raw);
                    if (alpha < kAlphaMin) continue;
                    any = true;
                    const float Tb = T[k] / (1.f - alpha);
                    const float w = alpha * Tb;
                    float dalpha = 0.f;
                    const float cc[3] = {r.col.x, r.col.y, r.col.z};
#pragma unroll
                    for (int c = 0; c < 3; ++c) {
                        acc[6 + c] = fmaf(w, dC[k][c], acc[6 + c]);
                        dalpha = fmaf(cc[c] - Bc[k][c], dC[k][c], dalpha);
                        Bc[k][c] = fmaf(alpha, cc[c] - Bc[k][c], Bc[k][c]);
                    }
                    dalpha *= Tb;
                    T[k] = Tb;
                    if (raw < kAlphaMax) {
                        acc[5] = fmaf(G, dalpha, acc[5]);
                        const float dp = alpha * dalpha;
                        const float ca = r.geo2.z, cb = r.geo2.w, cc2 = r.col.w;
                        acc[0] = fmaf(dp, ca * dx + cb * dy, acc[0]);
                        acc[1] = fmaf(dp, cb * dx + cc2 * dy, acc[1]);
                        acc[2] = fmaf(dp, -0.5f * dx * dx, acc[2]);
                        acc[3] = fmaf(dp, -dx * dy, acc[3]);
                        acc[4] = fmaf(dp, -0.5f * dy * dy, acc[4]);
                    }
                }
                if (__any_sync(kFull, any)) {
#pragma unroll
                    for (int c = 0; c < kPart; ++c) {
                        float v = acc[c];
#pragma unroll
                        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
                        acc[c] = v;
                    }
                    if (lane == 0) {
#pragma unroll
                        for (int c = 0; c < kPart; ++c) s_part[j][warp][c] = acc[c];
                    }
                }
            }
        }
        __syncthreads();
        // Block sum over warps in warp order, one record per pair.
        for (int e = threadIdx.x; e < cnt * kPart; e += THREADS) {
            const int j = e / kPart, c = e - j * kPart;
            float s = 0.f;
#pragma unroll
            for (int w = 0; w < WARPS; ++w) s += s_part[j][w][c];
            partials[(size_t)s_slot[j] * kPart + c] = s;
        }
    }
}

// Real SH basis of degree 3 (Condon-Shortley phase, index l*l + l + m) and
// its gradient with respect to the (unit) direction.
__device__ __forceinline__ void sh_basis_grad(float x, float y, float z, float* Y, float (*dY)[3]) {
    const float k0 = 0.28209479177387814f, k1 = 0.4886025119029199f;
    const float k2a = 1.0925484305920792f, k2b = 0.31539156525252005f, k2c = 0.5462742152960396f;
    const float k3a = 0.5900435899266435f, k3b = 2.890611442640554f, k3c = 0.4570457994644658f;
    const float k3d = 0.3731763325901154f, k3e = 1.445305721320277f;
    const float xx = x * x, yy = y * y, zz = z * z;
    Y[0] = k0;
    dY[0][0] = dY[0][1] = dY[0][2] = 0.f;
    Y[1] = -k1 * y;  dY[1][0] = 0.f; dY[1][1] = -k1; dY[1][2] = 0.f;
    Y[2] = k1 * z;   dY[2][0] = 0.f; dY[2][1] = 0.f; dY[2][2] = k1;
    Y[3] = -k1 * x;  dY[3][0] = -k1; dY[3][1] = 0.f; dY[3][2] = 0.f;
    Y[4] = k2a * x * y;  dY[4][0] = k2a * y; dY[4][1] = k2a * x; dY[4][2] = 0.f;
    Y[5] = -k2a * y * z; dY[5][0] = 0.f; dY[5][1] = -k2a * z; dY[5][2] = -k2a * y;
    Y[6] = k2b * (2.f * zz - xx - yy);
    dY[6][0] = -2.f * k2b * x; dY[6][1] = -2.f * k2b * y; dY[6][2] = 4.f * k2b * z;
    Y[7] = -k2a * x * z; dY[7][0] = -k2a * z; dY[7][1] = 0.f; dY[7][2] = -k2a * x;
    Y[8] = k2c * (xx - yy); dY[8][0] = 2.f * k2c * x; dY[8][1] = -2.f * k2c * y; dY[8][2] = 0.f;
    Y[9] = -k3a * y * (3.f * xx - yy);
    dY[9][0] = -6.f * k3a * x * y; dY[9][1] = -3.f * k3a * (xx - yy); dY[9][2] = 0.f;
    Y[10] = k3b * x * y * z;
    dY[10][0] = k3b * y * z; dY[10][1] = k3b * x * z; dY[10][2] = k3b * x * y;
    Y[11] = -k3c * y * (4.f * zz - xx - yy);
    dY[11][0] = 2.f * k3c * x * y; dY[11][1] = -k3c * (4.f * zz - xx - 3.f * yy); dY[11][2] = -8.f * k3c * y * z;
    Y[12] = k3d * z * (2.f * zz - 3.f * xx - 3.f * yy);
    dY[12][0] = -6.f * k3d * x * z; dY[12][1] = -6.f * k3d * y * z; dY[12][2] = k3d * (6.f * zz - 3.f * xx - 3.f * yy);
    Y[13] = -k3c * x * (4.f * zz - xx - yy);
    dY[13][0] = -k3c * (4.f * zz - 3.f * xx - yy); dY[13][1] = 2.f * k3c * x * y; dY[13][2] = -8.f * k3c * x * z;
    Y[14] = k3e * z * (xx - yy);
    dY[14][0] = 2.f * k3e * x * z; dY[14][1] = -2.f * k3e * y * z; dY[14][2] = k3e * (xx - yy);
    Y[15] = -k3a * x * (xx - 3.f * yy);
    dY[15][0] = -3.f * k3a * (xx - yy); dY[15][1] = 6.f * k3a * x * y; dY[15][2] = 0.f;
}

constexpr int kPbThreads = 128;
constexpr int kShPad = 52;

__global__ void __launch_bounds__(kPbThreads)
k_preprocess_bwd(int64_t n, const float* __restrict__ means, const float* __restrict__ log_scales,
                 const float4* __restrict__ quats, const float4* __restrict__ sh, const Frame f,
                 const float* __restrict__ rgb, const float* __restrict__ opacity,
                 const uint32_t* __restrict__ offsets, const uint32_t* __restrict__ touched,
                 const float* __restrict__ partials, float* __restrict__ d_means,
                 float* __restrict__ d_log_scales, float4* __restrict__ d_quats,
                 float* __restrict__ d_logits, float4* __restrict__ d_sh) {
    __shared__ __align__(16) float s_sh[kPbThreads / kWarp][kWarp * kShPad];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t i = (int64_t)blockIdx.x * kPbThreads + threadIdx.x;
    const bool valid = i < n;
    const uint32_t cnt = valid ? __ldg(touched + i) : 0u;
    const bool vis = cnt > 0;

    float gm[3] = {0.f, 0.f, 0.f}, gls[3] = {0.f, 0.f, 0.f}, gq[4] = {0.f, 0.f, 0.f, 0.f}, glogit = 0.f;
    float pr[kPart];
#pragma unroll
    for (int c = 0; c < kPart; ++c) pr[c] = 0.f;
    float X[3] = {0.f, 0.f, 0.f};
    if (vis) {
        // slot-ordered sum of this Gaussian's pair records
        const float* src = partials + (size_t)__ldg(offsets + i) * kPart;
        for (uint32_t s = 0; s < cnt; ++s)
#pragma unroll
            for (int c = 0; c < kPart; ++c) pr[c] += __ldg(src + s * kPart + c);
        X[0] = __ldg(means + 3 * i);
        X[1] = __ldg(means + 3 * i + 1);
        X[2] = __ldg(means + 3 * i + 2);
        const float sig = __ldg(opacity + i);
        glogit = pr[5] * sig * (1.f - sig);

        // forward quantities
        const float4 q4 = __ldg(quats + i);
        const float qn2 = q4.x * q4.x + q4.y * q4.y + q4.z * q4.z + q4.w * q4.w;
        const float qinv = rsqrtf(qn2);
        const float w = q4.x * qinv, x = q4.y * qinv, y = q4.z * qinv, z = q4.w * qinv;
        const float R[3][3] = {{1.f - 2.f * (y * y + z * z), 2.f * (x * y - w * z), 2.f * (x * z + w * y)},
                               {2.f * (x * y + w * z), 1.f - 2.f * (x * x + z * z), 2.f * (y * z - w * x)},
                               {2.f * (x * z - w * y), 2.f * (y * z + w * x), 1.f - 2.f * (x * x + y * y)}};
        const float s[3] = {expf(__ldg(log_scales + 3 * i)), expf(__ldg(log_scales + 3 * i + 1)),
                            expf(__ldg(log_scales + 3 * i + 2))};
        float M[3][3];
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int b = 0; b < 3; ++b) M[a][b] = R[a][b] * s[b];
        float t[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) t[a] = f.R[3 * a] * X[0] + f.R[3 * a + 1] * X[1] + f.R[3 * a + 2] * X[2] + f.t[a];
        const float rz = 1.f / t[2];
        const float rxu = t[0] * rz, ryu = t[1] * rz;
        const float rx = fminf(f.limx, fmaxf(-f.limx, rxu)), ry = fminf(f.limy, fmaxf(-f.limy, ryu));
        const bool clx = rx != rxu, cly = ry != ryu;
        const float j00 = f.fx * rz, j02 = -f.fx * rx * rz, j11 = f.fy * rz, j12 = -f.fy * ry * rz;
        float Tm[2][3];
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            Tm[0][b] = j00 * f.R[b] + j02 * f.R[6 + b];
            Tm[1][b] = j11 * f.R[3 + b] + j12 * f.R[6 + b];
        }
        // V = Tm M; Sigma' = V V^T + dilation I
        float V[2][3];
#pragma unroll
        for (int a = 0; a < 2; ++a)
#pragma unroll
            for (int k = 0; k < 3; ++k) V[a][k] = Tm[a][0] * M[0][k] + Tm[a][1] * M[1][k] + Tm[a][2] * M[2][k];
        const float sxx = V[0][0] * V[0][0] + V[0][1] * V[0][1] + V[0][2] * V[0][2] + f.dilation;
        const float sxy = V[0][0] * V[1][0] + V[0][1] * V[1][1] + V[0][2] * V[1][2];
        const float syy = V[1][0] * V[1][0] + V[1][1] * V[1][1] + V[1][2] * V[1][2] + f.dilation;

        // conic = Sigma'^{-1}: (a, b, c) = (syy, -sxy, sxx) / D
        const float D = fmaf(sxx, syy, -sxy * sxy), iD = 1.f / D, iD2 = iD * iD;
        const float ga = pr[2], gb = pr[3], gc = pr[4];
        const float gp = ga * (-syy * syy * iD2) + gb * (sxy * syy * iD2) + gc * (iD - sxx * syy * iD2);
        const float gs = ga * (iD - syy * sxx * iD2) + gb * (sxy * sxx * iD2) + gc * (-sxx * sxx * iD2);
        const float gr = ga * (2.f * sxy * syy * iD2) + gb * (-iD - 2.f * sxy * sxy * iD2) + gc * (2.f * sxy * sxx * iD2);
        const float G2[2][2] = {{gp, 0.5f * gr}, {0.5f * gr, gs}};
        // Sigma' = V V^T: dV = 2 G2 V; V = Tm M: dTm = dV M^T, dM = Tm^T dV
        float dV[2][3];
#pragma unroll
        for (int a = 0; a < 2; ++a)
#pragma unroll
            for (int k = 0; k < 3; ++k) dV[a][k] = 2.f * (G2[a][0] * V[0][k] + G2[a][1] * V[1][k]);
        float GT[2][3];
#pragma unroll
        for (int a = 0; a < 2; ++a)
#pragma unroll
            for (int b = 0; b < 3; ++b) GT[a][b] = dV[a][0] * M[b][0] + dV[a][1] * M[b][1] + dV[a][2] * M[b][2];
        // Tm = J W: dJ = GT W^T (entries 00, 02, 11, 12 are the live ones)
        const float gj00 = GT[0][0] * f.R[0] + GT[0][1] * f.R[1] + GT[0][2] * f.R[2];
        const float gj02 = GT[0][0] * f.R[6] + GT[0][1] * f.R[7] + GT[0][2] * f.R[8];
        const float gj11 = GT[1][0] * f.R[3] + GT[1][1] * f.R[4] + GT[1][2] * f.R[5];
        const float gj12 = GT[1][0] * f.R[6] + GT[1][1] * f.R[7] + GT[1][2] * f.R[8];
        const float rz2 = rz * rz;
        float gt[3] = {0.f, 0.f, 0.f};
        gt[2] += -gj00 * f.fx * rz2 - gj11 * f.fy * rz2;
        if (!clx) { gt[0] += -gj02 * f.fx * rz2; gt[2] += 2.f * gj02 * f.fx * rx * rz2; }
        else gt[2] += gj02 * f.fx * rx * rz2;
        if (!cly) { gt[1] += -gj12 * f.fy * rz2; gt[2] += 2.f * gj12 * f.fy * ry * rz2; }
        else gt[2] += gj12 * f.fy * ry * rz2;
        // projected centre m = (fx tx/tz + cx, fy ty/tz + cy)
        gt[0] += pr[0] * f.fx * rz;
        gt[1] += pr[1] * f.fy * rz;
        gt[2] -= (pr[0] * f.fx * t[0] + pr[1] * f.fy * t[1]) * rz2;
#pragma unroll
        for (int a = 0; a < 3; ++a) gm[a] = f.R[a] * gt[0] + f.R[3 + a] * gt[1] + f.R[6 + a] * gt[2];
        // M = R diag(s): dM = Tm^T dV
        float GR[3][3];
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            float dsb = 0.f;
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                const float gma = Tm[0][a] * dV[0][b] + Tm[1][a] * dV[1][b];
                dsb = fmaf(gma, R[a][b], dsb);
                GR[a][b] = gma * s[b];
            }
            gls[b] = dsb * s[b];
        }
        float gqh[4];
        gqh[0] = 2.f * (-z * GR[0][1] + y * GR[0][2] + z * GR[1][0] - x * GR[1][2] - y * GR[2][0] + x * GR[2][1]);
        gqh[1] = 2.f * (y * GR[0][1] + z * GR[0][2] + y * GR[1][0] - 2.f * x * GR[1][1] - w * GR[1][2] +
                        z * GR[2][0] + w * GR[2][1] - 2.f * x * GR[2][2]);
        gqh[2] = 2.f * (-2.f * y * GR[0][0] + x * GR[0][1] + w * GR[0][2] + x * GR[1][0] + z * GR[1][2] -
                        w * GR[2][0] + z * GR[2][1] - 2.f * y * GR[2][2]);
        gqh[3] = 2.f * (-2.f * z * GR[0][0] - w * GR[0][1] + x * GR[0][2] + w * GR[1][0] - 2.f * z * GR[1][1] +
                        y * GR[1][2] + x * GR[2][0] + y * GR[2][1]);
        const float qh[4] = {w, x, y, z};
        const float qd = gqh[0] * w + gqh[1] * x + gqh[2] * y + gqh[3] * z;
#pragma unroll
        for (int a = 0; a < 4; ++a) gq[a] = (gqh[a] - qd * qh[a]) * qinv;
    }

    // SH colour adjoint with warp-staged (coalesced) SH reads and gradient writes.
    const int64_t warp_first = (int64_t)blockIdx.x * kPbThreads + warp * kWarp;
    float* stage = s_sh[warp];
    const int64_t avail = n - warp_first;
    const int nvec = avail <= 0 ? 0 : (int)(avail >= kWarp ? kWarp * 12 : avail * 12);
    const bool any_vis = __any_sync(kFull, vis);
    if (any_vis) {
        const float4* src = sh + warp_first * 12;
#pragma unroll
        for (int r = 0; r < 12; ++r) {
            const int v = lane + r * kWarp;
            if (v < nvec) {
                const int g = v / 12, c = v - g * 12;
                *reinterpret_cast<float4*>(stage + g * kShPad + 4 * c) = __ldg(src + v);
            }
        }
        __syncwarp();
    }
    float* mine = stage + lane * kShPad;
    if (vis) {
        const float dx = X[0] - f.campos[0], dy = X[1] - f.campos[1], dz = X[2] - f.campos[2];
        const float invn = rsqrtf(dx * dx + dy * dy + dz * dz);
        const float d[3] = {dx * invn, dy * invn, dz * invn};
        float Y[16], dY[16][3];
        sh_basis_grad(d[0], d[1], d[2], Y, dY);
        float gd[3] = {0.f, 0.f, 0.f};
        float gcol[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) gcol[c] = __ldg(rgb + 3 * i + c) > 0.f ? pr[6 + c] : 0.f;
#pragma unroll
        for (int k = 0; k < 16; ++k) {
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const float coef = mine[3 * k + c];
                gd[0] = fmaf(coef * gcol[c], dY[k][0], gd[0]);
                gd[1] = fmaf(coef * gcol[c], dY[k][1], gd[1]);
                gd[2] = fmaf(coef * gcol[c], dY[k][2], gd[2]);
            }
        }
#pragma unroll
        for (int k = 0; k < 16; ++k)
#pragma unroll
            for (int c = 0; c < 3; ++c) mine[3 * k + c] = Y[k] * gcol[c];
        const float dd = gd[0] * d[0] + gd[1] * d[1] + gd[2] * d[2];
#pragma unroll
        for (int a = 0; a < 3; ++a) gm[a] += (gd[a] - dd * d[a]) * invn;
    } else if (any_vis) {
#pragma unroll
        for (int k = 0; k < 48; ++k) mine[k] = 0.f;
    }
    if (any_vis) {
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
                            const float* sh, const Frame& f, const float* mean2d, const float* conic,
                            const float* rgb, const float* opacity, const uint16_t* rect,
                            const uint32_t* offsets, const uint32_t* tiles_touched,
                            const uint32_t* vals, const uint32_t* ranges, const float* t_final,
                            const uint32_t* n_contrib, const float* d_image, float* d_means,
                            float* d_log_scales, float* d_quats, float* d_logits, float* d_sh,
                            void* scratch, cudaStream_t stream) {
    float* partials = static_cast<float*>(scratch);
    const int ntiles = f.TX * f.TY;
    const uint2* r2 = reinterpret_cast<const uint2*>(ranges);
    const float4* m4 = reinterpret_cast<const float4*>(mean2d);
    const uint2* rc = reinterpret_cast<const uint2*>(rect);
    if (ntiles > 0) {
        switch (f.TS) {
            case 8:
                k_blend_bwd<8><<<ntiles, 64, 0, stream>>>(r2, vals, m4, conic, opacity, rgb, rc, offsets, f,
                                                          t_final, n_contrib, d_image, partials);
                break;
            case 16:
                k_blend_bwd<16><<<ntiles, 256, 0, stream>>>(r2, vals, m4, conic, opacity, rgb, rc, offsets, f,
                                                            t_final, n_contrib, d_image, partials);
                break;
            case 32:
                k_blend_bwd<32><<<ntiles, 256, 0, stream>>>(r2, vals, m4, conic, opacity, rgb, rc, offsets, f,
                                                            t_final, n_contrib, d_image, partials);
                break;
            default:
                return cudaErrorInvalidValue;
        }
    }
    if (n > 0) {
        const int64_t blocks = (n + kPbThreads - 1) / kPbThreads;
        k_preprocess_bwd<<<(unsigned)blocks, kPbThreads, 0, stream>>>(
            n, means, log_scales, reinterpret_cast<const float4*>(quats), reinterpret_cast<const float4*>(sh), f,
            rgb, opacity, offsets, tiles_touched, partials, d_means, d_log_scales,
            reinterpret_cast<float4*>(d_quats), d_logits, reinterpret_cast<float4*>(d_sh));
    }
    return cudaGetLastError();
}

}  // namespace ws
