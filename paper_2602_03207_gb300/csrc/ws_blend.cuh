// Per-tile blend body (paper §3.4 with §2.1's compositing), shared by the
// single-view and the batched rasterisation kernels.
#pragma once

#include <type_traits>

#include "ws_common.cuh"

namespace ws {

constexpr int kBlendBatch = 256;

// Bitmask of the tile's BW x BH pixel blocks (BPR per row, BROWS rows) that
// a splat at tile-relative (x, y) can reach with alpha >= 1/255 (§3.4), i.e.
// whose pixel centres meet the bounding box of the ellipse
// q = a dx^2 + 2 b dx dy + c dy^2 <= qc: half-widths sqrt(qc Sigma'_xx),
// sqrt(qc Sigma'_yy) with Sigma' = [[c, -b], [-b, a]] / det. The box carries
// a margin (relative and absolute) well above the error of the approximate
// reciprocal and square roots, so no pixel that the blend's own test keeps is
// left out; a block visited without need adds w = 0.
template <int BW, int BH, int BPR, int BROWS>
__device__ __forceinline__ uint32_t splat_block_mask(float x, float y, float a, float b, float c, float qc) {
    const float rdet = rcp_approx(fmaf(a, c, -b * b));
    const float ex = sqrt_approx(qc * c * rdet) * 1.0001f + 1e-3f;
    const float ey = sqrt_approx(qc * a * rdet) * 1.0001f + 1e-3f;
    return box_block_mask<BW, BH, BPR, BROWS>(x - ex, x + ex, y - ey, y + ey);
}

// Shared-memory record of one splat for the blend (48 bytes).
struct SplatRec {
    float4 geo;   // tile-relative centre x, y; conic premultiplied A, B
    float4 geo2;  // C, log2(opacity), -, -
    float4 col;   // r, g, b, -
};

// Per-splat inputs of the blend, read from the splat records of
// ws_preprocess (three 16-byte loads of one 48-byte record): the double-float
// centre (made tile-relative without large-magnitude rounding), the conic
// (a, b, c), sigma and the colour.
struct FloatSplats {
    const float4* __restrict__ rec;
    __device__ __forceinline__ void load(uint32_t g, float ox, float oy, float& x, float& y, float& a, float& b,
                                         float& c, float& op, float4& col) const {
        const float4 m = __ldg(rec + kSplatVec4 * g);
        const float4 k = __ldg(rec + kSplatVec4 * g + 1);
        col = __ldg(rec + kSplatVec4 * g + 2);
        x = __fadd_rn(__fsub_rn(m.x, ox), m.z);
        y = __fadd_rn(__fsub_rn(m.y, oy), m.w);
        a = k.x;
        b = k.y;
        c = k.z;
        op = k.w;
    }
};

// Bitmask of a tile's 4x4 pixel sub-blocks (SPR per row and per column, bit
// row * SPR + col) whose pixel centres meet the box [xl, xh] x [yl, yh].
template <int SPR, typename MaskT>
__device__ __forceinline__ MaskT box_subblock_mask(float xl, float xh, float yl, float yh) {
    MaskT cols = 0;
#pragma unroll
    for (int c = 0; c < SPR; ++c)
        cols |= (xl <= (float)(c * 4) + 3.5f && xh >= (float)(c * 4) + 0.5f) ? (MaskT(1) << c) : MaskT(0);
    MaskT mask = 0;
#pragma unroll
    for (int r = 0; r < SPR; ++r)
        mask |= (yl <= (float)(r * 4) + 3.5f && yh >= (float)(r * 4) + 0.5f) ? (cols << (r * SPR)) : MaskT(0);
    return mask;
}

template <int SPR, typename MaskT>
__device__ __forceinline__ MaskT splat_subblock_mask(float x, float y, float a, float b, float c, float qc) {
    const float rdet = rcp_approx(fmaf(a, c, -b * b));
    const float ex = sqrt_approx(qc * c * rdet) * 1.0001f + 1e-3f;
    const float ey = sqrt_approx(qc * a * rdet) * 1.0001f + 1e-3f;
    return box_subblock_mask<SPR, MaskT>(x - ex, x + ex, y - ey, y + ey);
}

template <int TS>
struct SubMask {
    using T = typename std::conditional<((TS / 4) * (TS / 4) > 32), unsigned long long, uint32_t>::type;
};

// One block per tile. Each warp owns WPB (TS^2/256, at least 1) 8x4 pixel
// regions, each split into two 4x4 sub-blocks, one per half-warp. Splats are
// staged 256 at a time; while staging, every splat also records the bitmask
// of the tile's 4x4 sub-blocks that the bounding box of its opacity-aware
// ellipse meets. Each half-warp then walks the batch 32 splats at a time and
// visits only the splats of its own sub-block, in list order; the two halves
// run in lockstep for max(visits of either half) steps, the idle half adding
// w = 0, so per pixel the compositing order and arithmetic are unchanged.
template <int TS, typename Splats>
__device__ __forceinline__ void blend_tile(const Frame& f, int tile, uint2 range, const uint32_t* __restrict__ vals,
                                           const Splats& sp, float* __restrict__ image, float* __restrict__ t_final,
                                           uint32_t* __restrict__ n_contrib) {
    constexpr int THREADS = TS * TS >= 256 ? 256 : TS * TS;
    constexpr int WARPS = THREADS / 32;
    constexpr int PPT = TS * TS / THREADS;  // 8x4 regions per warp (TS = 32: 4)
    constexpr int RPR = TS / 8;             // regions per row
    constexpr int SPR = TS / 4;             // sub-blocks per row
    using MaskT = typename SubMask<TS>::T;
    __shared__ SplatRec s_rec[kBlendBatch];
    __shared__ MaskT s_mask[kBlendBatch];

    const int tx = tile % f.TX, ty = tile / f.TX;
    const float ox = (float)(tx * TS), oy = (float)(ty * TS);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int half = lane >> 4;

    float px[PPT], py[PPT], T[PPT], C0[PPT], C1[PPT], C2[PPT];
    uint32_t last[PPT];
    int sba[PPT];
#pragma unroll
    for (int k = 0; k < PPT; ++k) {
        const int rg = warp + k * WARPS;
        const int rx = rg % RPR, ry = rg / RPR;
        px[k] = (float)(rx * 8 + half * 4 + (lane & 3)) + 0.5f;
        py[k] = (float)(ry * 4 + ((lane >> 2) & 3)) + 0.5f;
        sba[k] = ry * SPR + 2 * rx;
        T[k] = 1.f;
        C0[k] = C1[k] = C2[k] = 0.f;
        last[k] = 0;
    }

    for (uint32_t start = range.x; start < range.y; start += kBlendBatch) {
        const int cnt = (int)min((uint32_t)kBlendBatch, range.y - start);
        __syncthreads();
        for (int j = threadIdx.x; j < cnt; j += THREADS) {
            const uint32_t g = __ldg(vals + start + j);
            float a, b, c, op;
            SplatRec r;
            sp.load(g, ox, oy, r.geo.x, r.geo.y, a, b, c, op, r.col);
            r.geo.z = -0.5f * kLog2e * a;
            r.geo.w = -kLog2e * b;
            const float L = lg2_approx(op);
            r.geo2 = make_float4(-0.5f * kLog2e * c, L, 0.f, 0.f);
            s_rec[j] = r;
            const float qc = (f.flags & WS_CFG_FIXED_RADIUS) ? 2.f * kLn255 : fmaxf(0.f, kTwoLn2 * (L - kLog2AlphaMin));
            s_mask[j] = splat_subblock_mask<SPR, MaskT>(r.geo.x, r.geo.y, a, b, c, qc);
        }
        __syncthreads();
        const uint32_t rel = start + 1 - range.x;
#pragma unroll
        for (int k = 0; k < PPT; ++k) {
            for (int base = 0; base < cnt; base += 32) {
                const int jj = base + lane;
                const MaskT m = jj < cnt ? s_mask[jj] : MaskT(0);
                const uint32_t ba = __ballot_sync(kFull, (uint32_t)(m >> sba[k]) & 1u);
                const uint32_t bb = __ballot_sync(kFull, (uint32_t)(m >> (sba[k] + 1)) & 1u);
                uint32_t bits = half ? bb : ba;
                const int steps = max(__popc(ba), __popc(bb));
                for (int it = 0; it < steps; ++it) {
                    // The idle half (no splat left) re-reads entry `base` and
                    // adds w = 0, which leaves C and T bit for bit unchanged.
                    const bool act = bits != 0u;
                    const int j = base + (act ? __ffs(bits) - 1 : 0);
                    bits &= bits - 1u;
                    const float4 geo = s_rec[j].geo;
                    const float2 geo2 = *reinterpret_cast<const float2*>(&s_rec[j].geo2);
                    const float dx = px[k] - geo.x, dy = py[k] - geo.y;
                    const float e = splat_log2_alpha(dx, dy, geo.z, geo.w, geo2.x, geo2.y);
                    const bool keep = act && e >= kLog2AlphaMin;
                    const float alpha = fminf(kAlphaMax, ex2_approx(e));
                    const float w = keep ? alpha * T[k] : 0.f;
                    const float4 col = s_rec[j].col;
                    C0[k] = fmaf(col.x, w, C0[k]);
                    C1[k] = fmaf(col.y, w, C1[k]);
                    C2[k] = fmaf(col.z, w, C2[k]);
                    T[k] = T[k] - w;
                    last[k] = keep ? rel + j : last[k];
                }
            }
        }
    }

#pragma unroll
    for (int k = 0; k < PPT; ++k) {
        const int gx = tx * TS + (int)px[k], gy = ty * TS + (int)py[k];
        if (gx < f.W && gy < f.H) {
            const size_t pix = (size_t)gy * f.W + gx;
            image[3 * pix] = fmaf(T[k], f.bg[0], C0[k]);
            image[3 * pix + 1] = fmaf(T[k], f.bg[1], C1[k]);
            image[3 * pix + 2] = fmaf(T[k], f.bg[2], C2[k]);
            t_final[pix] = T[k];
            n_contrib[pix] = last[k];
        }
    }
}


constexpr int kBwdBatch = 64;
constexpr int kPart = 9;  // dmean x, y; dconic a, b, c; sigma dsigma; drgb r, g, b

struct BwdRec {
    float4 geo;   // tile-relative centre x, y; premultiplied conic A, B
    float4 geo2;  // premultiplied C, log2(opacity), conic a, conic b
    float4 col;   // r, g, b, conic c
};

// `tile` is the tile index within the frame; `slot_of(g)` gives the first
// emission slot of Gaussian g's pairs for this frame (offsets[g] for one view,
// offsets[g * views + v] in a batch).
template <int TS, typename SlotBase>
__device__ __forceinline__ void blend_bwd_tile(const Frame& f, int tile, uint2 range, const uint32_t* __restrict__ vals,
                                               const float4* __restrict__ splats, const uint2* __restrict__ rect,
                                               SlotBase slot_of,
                                               const float* __restrict__ t_final,
                                               const uint32_t* __restrict__ n_contrib,
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

    const int tx = tile % f.TX, ty = tile / f.TX;
    const float ox = (float)(tx * TS), oy = (float)(ty * TS);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
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
        const uint32_t slot = slot_of(g) + (ty - y0) * (x1 - x0 + 1) + (tx - x0);
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
            const float4 m = __ldg(splats + kSplatVec4 * g);
            const float4 k = __ldg(splats + kSplatVec4 * g + 1);
            const float4 cl = __ldg(splats + kSplatVec4 * g + 2);
            const float a = k.x, b = k.y, c = k.z, op = k.w;
            BwdRec r;
            r.geo.x = __fadd_rn(__fsub_rn(m.x, ox), m.z);
            r.geo.y = __fadd_rn(__fsub_rn(m.y, oy), m.w);
            r.geo.z = -0.5f * kLog2e * a;
            r.geo.w = -kLog2e * b;
            const float L = lg2_approx(op);
            r.geo2 = make_float4(-0.5f * kLog2e * c, L, a, b);
            r.col = make_float4(cl.x, cl.y, cl.z, c);
            s_rec[j] = r;
            const float qc = (f.flags & WS_CFG_FIXED_RADIUS) ? 2.f * kLn255 : fmaxf(0.f, kTwoLn2 * (L - kLog2AlphaMin));
            s_mask[j] = splat_block_mask<BW, BH, BPR, BROWS>(r.geo.x, r.geo.y, a, b, c, qc);
            const uint2 rc = __ldg(rect + g);
            const uint32_t x0 = rc.x & 0xffffu, y0 = rc.x >> 16, x1 = rc.y & 0xffffu;
            s_slot[j] = slot_of(g) + (ty - y0) * (x1 - x0 + 1) + (tx - x0);
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
                    const float e = splat_log2_alpha(dx, dy, r.geo.z, r.geo.w, r.geo2.x, r.geo2.y);
                    if (!(e >= kLog2AlphaMin)) continue;
                    const float raw = ex2_approx(e);
                    const float alpha = fminf(kAlphaMax, raw);
                    any = true;
                    // T before this pair, T_after / (1 - alpha), with the
                    // reciprocal on the special-function unit (a few ulp;
                    // 1 - alpha >= 0.01)
                    const float Tb = T[k] * rcp_approx(1.f - alpha);
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
                        // partial 5 is sigma dL/dsigma = raw dL/dalpha
                        // (d alpha / d sigma = exp(-q/2) = raw / sigma)
                        acc[5] = fmaf(raw, dalpha, acc[5]);
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
                    // Warp sums of the 9 partials in a fixed order with 14
                    // shuffles: partials 0..7 by reduce-scatter (each step
                    // hands half of a lane's values to its partner, so after
                    // offsets 16, 8, 4 lane l holds partial (l >> 2) & 7
                    // summed over 8 lanes, then two butterfly steps finish
                    // it), partial 8 by a butterfly.
                    const bool b4 = lane & 16, b3 = lane & 8, b2 = lane & 4;
                    float h4[4];
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const float give = b4 ? acc[q] : acc[4 + q];
                        const float keep = b4 ? acc[4 + q] : acc[q];
                        h4[q] = keep + __shfl_xor_sync(kFull, give, 16);
                    }
                    float h2[2];
#pragma unroll
                    for (int q = 0; q < 2; ++q) {
                        const float give = b3 ? h4[q] : h4[2 + q];
                        const float keep = b3 ? h4[2 + q] : h4[q];
                        h2[q] = keep + __shfl_xor_sync(kFull, give, 8);
                    }
                    float h1 = (b2 ? h2[1] : h2[0]) + __shfl_xor_sync(kFull, b2 ? h2[0] : h2[1], 4);
                    h1 += __shfl_xor_sync(kFull, h1, 2);
                    h1 += __shfl_xor_sync(kFull, h1, 1);
                    float v8 = acc[8];
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) v8 += __shfl_xor_sync(kFull, v8, o);
                    if ((lane & 3) == 0) s_part[j][warp][lane >> 2] = h1;
                    if (lane == 0) s_part[j][warp][8] = v8;
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

}  // namespace ws
