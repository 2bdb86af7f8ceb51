// Per-tile blend bodies (paper §3.4 with §2.1's compositing) shared by the
// single-view, batched and fused training kernels: the forward composite,
// its deterministic adjoint, and both in one pass over a tile.
#pragma once

#include <type_traits>

#include "ws_common.cuh"

namespace ws {

constexpr int kBlendBatch = 256;  // splats staged in shared memory at a time
constexpr int kBwdChunk = 64;     // splats whose partials the backward holds at a time
// The fused training pass holds the partials of 32 splats at a time: half the
// partial buffer and 48 registers instead of 64 let five of its blocks share
// an SM instead of four.
constexpr int kTrainChunk = 32;
constexpr int kPart = 9;          // dmean x, y; dconic a, b, c; sigma dsigma; drgb r, g, b

// Blocks per SM that the forward blends are compiled for (their register
// budget): 64 threads x 16, 256 x 8 and 1024 x 2 for 8, 16 and 32 pixel
// tiles (one thread per pixel).
template <int TS>
constexpr int blend_min_blocks() { return TS == 8 ? 16 : (TS == 16 ? 8 : 2); }

// Shared-memory record of one staged splat (48 bytes):
//   geo  = tile-relative centre x, y; conic premultiplied A = -log2(e) a / 2,
//          B = -log2(e) b
//   geo2 = C = -log2(e) c / 2, L = log2(sigma); the splat's axis basis
//          e1 = (ct, st) (axis_basis; staged for the backward only)
//   col  = r, g, b; 0
// The forward reads geo, geo2.xy and col.xyz; the backward everything.
struct SplatRec {
    float4 geo;
    float4 geo2;
    float4 col;
};

// Staged records sit in groups of 33: slot 33 g holds a null splat (zero
// conic, L = -inf, so its log-alpha is -inf and it is never composited) and
// slots 33 g + 1 .. 33 g + 32 the splats 32 g .. 32 g + 31, so that a
// half-warp with nothing left to visit in a group of 32 reads the null splat
// at index 0 of the group (__ffs of an empty bit set) and needs no select.
__device__ __forceinline__ int rec_slot(int j) { return j + (j >> 5) + 1; }
__host__ __device__ constexpr int rec_slots(int batch) { return batch + batch / 32 + 1; }

// Writes the null splat of every group of a staging area of `batch` splats.
__device__ __forceinline__ void init_null_splats(SplatRec* s_rec, int batch) {
    for (int g = threadIdx.x; g <= (batch - 1) / 32; g += blockDim.x) {
        s_rec[33 * g].geo = make_float4(0.f, 0.f, 0.f, 0.f);
        s_rec[33 * g].geo2 = make_float4(0.f, -INFINITY, 0.f, 0.f);
        s_rec[33 * g].col = make_float4(0.f, 0.f, 0.f, 0.f);
    }
}

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

// Geometry of a TS x TS tile: TH threads, one per pixel of one 8x4 region per
// warp (PPT regions per warp when the tile has more pixels than threads);
// each region is two 4x4 sub-blocks, one per half-warp. A splat's mask has
// one bit per sub-block (row-major, SPR per row). The backward and the fused
// training pass take at most 256 threads (their per-half-warp partial
// buffers grow with the warps); the forward blend takes one thread per pixel.
template <int TS, int TH = (TS * TS >= 256 ? 256 : TS * TS)>
struct TileGeom {
    static constexpr int THREADS = TH;
    static constexpr int WARPS = THREADS / 32;
    static constexpr int PPT = TS * TS / THREADS;
    static constexpr int RPR = TS / 8;  // regions per row
    static constexpr int SPR = TS / 4;  // sub-blocks per row
    using Mask = typename std::conditional<(SPR * SPR > 32), unsigned long long, uint32_t>::type;
    // region k of this warp: lane's pixel (tile-relative, centre) and the
    // index of the region's left sub-block
    __device__ static __forceinline__ void pixel(int warp, int lane, int k, float& px, float& py, int& sb) {
        const int rg = warp + k * WARPS;
        const int rx = rg % RPR, ry = rg / RPR;
        px = (float)(rx * 8 + (lane >> 4) * 4 + (lane & 3)) + 0.5f;
        py = (float)(ry * 4 + ((lane >> 2) & 3)) + 0.5f;
        sb = ry * SPR + 2 * rx;
    }
};

// Bitmask of a tile's 4x4 sub-blocks whose pixel centres meet the box
// [xl, xh] x [yl, yh] (tile-relative): one compare pair per sub-block column
// and per sub-block row.
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

// Sub-blocks of columns [c_lo, c_hi] (clamped into [0, SPR)) as SPR bits:
// c_lo = ceil((xl - 3.5) / 4), c_hi = floor((xh - 0.5) / 4), the columns
// whose pixel centres 4c + 0.5 .. 4c + 3.5 meet [xl, xh].
template <int SPR>
__device__ __forceinline__ uint32_t span_bits(float xl, float xh) {
    const int lo = (int)ceilf(fmaxf((xl - 3.5f) * 0.25f, 0.f));
    const int hi = (int)floorf(fminf((xh - 0.5f) * 0.25f, (float)(SPR - 1)));
    return lo <= hi ? (2u << hi) - (1u << lo) : 0u;
}

// Bitmask of a tile's 4x4 sub-blocks that the ellipse q(dx, dy) =
// a dx^2 + 2 b dx dy + c dy^2 <= qm around the tile-relative centre (gx, gy)
// meets, one row of sub-blocks (a band of 4 pixel rows) at a time. Within
// the band the ellipse's dy runs over [u0, u1] (the band cut to the
// ellipse's half-height ey) and at height dy its x range is
// gx + (-b dy -/+ s(dy)) / a with s(dy) = sqrt(a qm - det dy^2); the left end
// is convex in dy and smallest at dy = b sqrt(qm / (det c)), the right end
// concave and largest at the opposite dy, so the band's x range is those two
// ends with dy clamped into [u0, u1]. The part of the ellipse in the band is
// convex, so it meets a sub-block of the band exactly when its x range meets
// the sub-block's columns.
template <int SPR, typename MaskT>
__device__ __forceinline__ MaskT ellipse_subblock_mask(float gx, float gy, float a, float b, float c, float qm,
                                                       float rdet, float ey, float xmargin) {
    const int r_lo = (int)ceilf(fmaxf((gy - ey - 3.5f) * 0.25f, 0.f));
    const int r_hi = (int)floorf(fminf((gy + ey - 0.5f) * 0.25f, (float)(SPR - 1)));
    const float det = fmaf(a, c, -b * b);
    const float aq = a * qm;
    const float ra = rcp_approx(a);
    const float dys = b * sqrt_approx(qm * rdet * rcp_approx(c));
    MaskT mask = 0;
    for (int r = r_lo; r <= r_hi; ++r) {
        const float u0 = fmaxf((float)(4 * r) + 0.5f - gy, -ey);
        const float u1 = fminf((float)(4 * r) + 3.5f - gy, ey);
        const float dl = fminf(fmaxf(dys, u0), u1);
        const float dr = fminf(fmaxf(-dys, u0), u1);
        const float sl = sqrt_approx(fmaxf(0.f, fmaf(-det, dl * dl, aq)));
        const float sr = sqrt_approx(fmaxf(0.f, fmaf(-det, dr * dr, aq)));
        const float xl = gx - fmaf(b, dl, sl) * ra - xmargin;
        const float xh = gx + fmaf(-b, dr, sr) * ra + xmargin;
        mask |= MaskT(span_bits<SPR>(xl, xh)) << (r * SPR);
    }
    return mask;
}

// Builds the staged record of one splat and the mask of the sub-blocks that
// its opacity-aware ellipse (§3.4) q = a dx^2 + 2 b dx dy + c dy^2 <= qc
// reaches: with ELLIPSE the sub-blocks that the ellipse itself meets
// (ellipse_subblock_mask), else those that its bounding box meets (half-
// widths sqrt(qc Sigma'_xx), sqrt(qc Sigma'_yy) with Sigma' = [[c, -b],
// [-b, a]] / det). The ellipse is grown to qm = 1.001 qc + 1e-3 and the
// ranges by a relative and an absolute margin, well above the error of the
// approximate reciprocal and square roots, so no pixel inside the exact
// ellipse is left out; a sub-block visited without need adds w = 0. The
// ellipse's mask costs more arithmetic per staged splat and saves visits
// (13 % of them on the 1080p / 1M frame): a gain where a visit is dear (the
// backward), not in the forward. WS_CFG_BOX_MASKS takes the box's mask
// everywhere; the results are the same bits either way.
template <int TS, bool ELLIPSE, typename Splats>
__device__ __forceinline__ void stage_splat(const Frame& f, float ox, float oy, const Splats& sp, uint32_t g,
                                            SplatRec* dst, typename TileGeom<TS>::Mask& mask) {
    float a, b, c, op, gx, gy;
    float4 col;
    sp.load(g, ox, oy, gx, gy, a, b, c, op, col);
    const float L = lg2_approx(op);
    // the record first: its registers are free before the mask's arithmetic
    float ct = 0.f, st = 0.f;
    if (ELLIPSE) axis_basis(col.w, ct, st);
    dst->geo = make_float4(gx, gy, -0.5f * kLog2e * a, -kLog2e * b);
    dst->geo2 = make_float4(-0.5f * kLog2e * c, L, ct, st);
    dst->col = make_float4(col.x, col.y, col.z, 0.f);
    const float qc = (f.flags & WS_CFG_FIXED_RADIUS) ? 2.f * kLn255 : fmaxf(0.f, kTwoLn2 * (L - kLog2AlphaMin));
    const float qm = fmaf(qc, 1.001f, 1e-3f);
    const float rdet = rcp_approx(fmaf(a, c, -b * b));
    const float ex = sqrt_approx(qm * c * rdet) * 1.0001f + 1e-3f;
    const float ey = sqrt_approx(qm * a * rdet) * 1.0001f + 1e-3f;
    using M = typename TileGeom<TS>::Mask;
    if (ELLIPSE && !(f.flags & WS_CFG_BOX_MASKS))
        mask = ellipse_subblock_mask<TileGeom<TS>::SPR, M>(gx, gy, a, b, c, qm, rdet, ey, fmaf(ex, 1e-4f, 1e-3f));
    else
        mask = box_subblock_mask<TileGeom<TS>::SPR, M>(gx - ex, gx + ex, gy - ey, gy + ey);
}

// Forward state of a thread's pixels: front to back, C += c a T, T -= a T.
template <int TS, int TH = TileGeom<TS>::THREADS>
struct FwdPixels {
    using G = TileGeom<TS, TH>;
    float px[G::PPT], py[G::PPT], T[G::PPT], C0[G::PPT], C1[G::PPT], C2[G::PPT];
    uint32_t last[G::PPT];
    int sb[G::PPT];

    __device__ __forceinline__ void init(int warp, int lane) {
#pragma unroll
        for (int k = 0; k < G::PPT; ++k) {
            G::pixel(warp, lane, k, px[k], py[k], sb[k]);
            T[k] = 1.f;
            C0[k] = C1[k] = C2[k] = 0.f;
            last[k] = 0;
        }
    }

    // Composites the staged splats [0, cnt) (list positions rel0 - 1 + j, made
    // 1-based for n_contrib). Each half-warp walks the batch 32 splats at a
    // time and visits only the splats whose mask has its own sub-block, in
    // list order; the two halves run in lockstep for max(visits of either
    // half) steps, the idle half visiting its group's null splat (w = 0,
    // which leaves C and T bit for bit unchanged), so per pixel the
    // compositing order and arithmetic are those of a plain front-to-back
    // loop. The last composited position is noted per group (1-based within
    // the group) and made a list position once at the group's end.
    __device__ __forceinline__ void batch(const SplatRec* s_rec, const typename G::Mask* s_mask, int cnt,
                                          uint32_t rel0, int lane) {
        const int half = lane >> 4;
#pragma unroll
        for (int k = 0; k < G::PPT; ++k) {
            for (int base = 0; base < cnt; base += 32) {
                const int jj = base + lane;
                const typename G::Mask m = jj < cnt ? s_mask[jj] : typename G::Mask(0);
                const uint32_t ba = __ballot_sync(kFull, (uint32_t)(m >> sb[k]) & 1u);
                const uint32_t bb = __ballot_sync(kFull, (uint32_t)(m >> (sb[k] + 1)) & 1u);
                uint32_t bits = half ? bb : ba;
                const int steps = max(__popc(ba), __popc(bb));
                const SplatRec* grp = s_rec + base + (base >> 5);  // grp[0]: the null splat
                int lastk = 0;
#pragma unroll 4
                for (int it = 0; it < steps; ++it) {
                    const int q = __ffs(bits);  // 0 once this half has no visit left
                    bits &= bits - 1u;
                    const float4 geo = grp[q].geo;
                    const float2 geo2 = *reinterpret_cast<const float2*>(&grp[q].geo2);
                    const float dx = px[k] - geo.x, dy = py[k] - geo.y;
                    const float e = splat_log2_alpha(dx, dy, geo.z, geo.w, geo2.x, geo2.y);
                    const bool keep = e >= kLog2AlphaMin;
                    const float alpha = fminf(kAlphaMax, ex2_approx(e));
                    const float w = keep ? alpha * T[k] : 0.f;
                    const float4 col = grp[q].col;
                    C0[k] = fmaf(col.x, w, C0[k]);
                    C1[k] = fmaf(col.y, w, C1[k]);
                    C2[k] = fmaf(col.z, w, C2[k]);
                    T[k] = T[k] - w;
                    lastk = keep ? q : lastk;
                }
                if (lastk) last[k] = rel0 + (uint32_t)(base + lastk - 1);
            }
        }
    }
};

// Backward state of a thread's pixels, walked back to front from the final
// transmittance. With B = colour behind the splat normalised by the
// transmittance after it (B starts as the background, B <- a c + (1 - a) B):
//   dL/dc = a T dL/dC,   dL/da = T (c - B) . dL/dC,
// and, unless the alpha was clamped at 0.99, sigma dL/dsigma = raw dL/da
// (raw = sigma G, the unclamped alpha) and dL/dpower = a dL/da with
// power = -1/2 d^T Q d, giving d/dmean = Q d, d/dQ_a = -dx^2/2,
// d/dQ_b = -dx dy, d/dQ_c = -dy^2/2.
template <int TS, int CHUNK = kBwdChunk>
struct BwdPixels {
    using G = TileGeom<TS>;
    float px[G::PPT], py[G::PPT], T[G::PPT], dC[G::PPT][3], Bc[G::PPT][3];
    uint32_t last[G::PPT];
    int sb[G::PPT];
    typename G::Mask wmask;  // sub-blocks of this warp's regions

    __device__ __forceinline__ void init_geometry(int warp, int lane) {
        wmask = 0;
#pragma unroll
        for (int k = 0; k < G::PPT; ++k) {
            G::pixel(warp, lane, k, px[k], py[k], sb[k]);
            wmask |= typename G::Mask(3) << sb[k];
        }
    }

    // Walks the staged splats [0, cnt) back to front (list positions pos0 +
    // j), in chunks of CHUNK. Each half-warp visits, back to front, the
    // splats whose mask has its own 4x4 sub-block; the two halves run in
    // lockstep for max(visits of either half) steps (an idle half evaluates
    // nothing). Each half sums its splat's 9 partials over its 16 pixels in
    // a fixed order and stores them in s_part[j][half-warp]; the block then
    // adds the half-warps that wrote, in order, and writes one record per
    // pair at its emission slot.
    __device__ __forceinline__ void batch(const SplatRec* s_rec, const typename G::Mask* s_mask,
                                          const uint32_t* s_slot, float (*s_part)[2 * G::WARPS][kPart],
                                          uint32_t* s_wrote, int cnt, uint32_t pos0, int warp, int lane,
                                          float* __restrict__ partials) {
        const int half = lane >> 4;
        const int hw = 2 * warp + half;  // this lane's half-warp
        for (int hi = cnt; hi > 0; hi -= CHUNK) {
            const int lo = max(0, hi - CHUNK);
            for (int j = threadIdx.x; j < hi - lo; j += G::THREADS) s_wrote[j] = 0u;
            __syncthreads();
#pragma unroll
            for (int k = 0; k < G::PPT; ++k) {
                for (int base = lo + (((hi - lo - 1) >> 5) << 5); base >= lo; base -= 32) {
                    const int jj = base + lane;
                    const typename G::Mask mm = jj < hi ? s_mask[jj] : typename G::Mask(0);
                    const uint32_t ba = __ballot_sync(kFull, (uint32_t)(mm >> sb[k]) & 1u);
                    const uint32_t bb = __ballot_sync(kFull, (uint32_t)(mm >> (sb[k] + 1)) & 1u);
                    uint32_t bits = half ? bb : ba;
                    const int steps = max(__popc(ba), __popc(bb));
                    for (int it = 0; it < steps; ++it) {
                        const bool act = bits != 0u;
                        const int hb = act ? 31 - __clz(bits) : 0;
                        bits &= ~(1u << hb);
                        const int j = base + hb;
                        const uint32_t pos = pos0 + (uint32_t)j;
                        float acc[kPart];
#pragma unroll
                        for (int c = 0; c < kPart; ++c) acc[c] = 0.f;
                        bool any = false;
                        if (act && pos < last[k]) {
                            const SplatRec r = s_rec[rec_slot(j)];
                            const float dx = px[k] - r.geo.x, dy = py[k] - r.geo.y;
                            const float e = splat_log2_alpha(dx, dy, r.geo.z, r.geo.w, r.geo2.x, r.geo2.y);
                            if (e >= kLog2AlphaMin) {
                                const float raw = ex2_approx(e);
                                const float alpha = fminf(kAlphaMax, raw);
                                any = true;
                                const float Tb = T[k] * rcp_approx(1.f - alpha);
                                const float w = alpha * Tb;
                                float dalpha = 0.f;
                                const float cc[3] = {r.col.x, r.col.y, r.col.z};
#pragma unroll
                                for (int c = 0; c < 3; ++c) {
                                    acc[6 + c] = w * dC[k][c];
                                    dalpha = fmaf(cc[c] - Bc[k][c], dC[k][c], dalpha);
                                    Bc[k][c] = fmaf(alpha, cc[c] - Bc[k][c], Bc[k][c]);
                                }
                                dalpha *= Tb;
                                T[k] = Tb;
                                if (raw < kAlphaMax) {
                                    acc[5] = raw * dalpha;
                                    const float dp = alpha * dalpha;
                                    // d/dmean = dp C d with C = -(2A, B; B, 2C) / log2(e)
                                    const float dpl = -kLn2 * dp;
                                    acc[0] = dpl * fmaf(2.f * r.geo.z, dx, r.geo.w * dy);
                                    acc[1] = dpl * fmaf(r.geo.w, dx, 2.f * r.geo2.x * dy);
                                    // conic derivatives in the splat's axis basis
                                    const float ct = r.geo2.z, st = r.geo2.w;
                                    const float u = fmaf(ct, dx, st * dy), v = fmaf(ct, dy, -st * dx);
                                    const float hdp = -0.5f * dp;
                                    acc[2] = hdp * (u * u);
                                    acc[3] = -dp * (u * v);
                                    acc[4] = hdp * (v * v);
                                }
                            }
                        }
                        const uint32_t anyb = __ballot_sync(kFull, any);
                        if (anyb) {
                            // Sums over each half's 16 lanes in a fixed order, 12
                            // shuffles for both halves: partials 0..7 by
                            // reduce-scatter (offsets 8, 4, 2; lane l of a half then
                            // holds partial (l >> 1) & 7 over 8 lanes) and a last
                            // butterfly step (offset 1), partial 8 by a butterfly.
                            const bool b3 = lane & 8, b2 = lane & 4, b1 = lane & 2;
                            float h4[4];
#pragma unroll
                            for (int q = 0; q < 4; ++q) {
                                const float give = b3 ? acc[q] : acc[4 + q];
                                const float keep = b3 ? acc[4 + q] : acc[q];
                                h4[q] = keep + __shfl_xor_sync(kFull, give, 8);
                            }
                            float h2[2];
#pragma unroll
                            for (int q = 0; q < 2; ++q) {
                                const float give = b2 ? h4[q] : h4[2 + q];
                                const float keep = b2 ? h4[2 + q] : h4[q];
                                h2[q] = keep + __shfl_xor_sync(kFull, give, 4);
                            }
                            float h1 = (b1 ? h2[1] : h2[0]) + __shfl_xor_sync(kFull, b1 ? h2[0] : h2[1], 2);
                            h1 += __shfl_xor_sync(kFull, h1, 1);
                            float v8 = acc[8];
#pragma unroll
                            for (int o = 8; o > 0; o >>= 1) v8 += __shfl_xor_sync(kFull, v8, o);
                            const bool mine = (anyb >> (16 * half)) & 0xffffu;  // this half has a partial
                            if (mine) {
                                // with several regions per warp, a half-warp adds to
                                // what it stored for the same splat in an earlier region
                                const bool add = G::PPT > 1 && ((s_wrote[j - lo] >> hw) & 1u);
                                const int p = ((lane & 15) >> 1);
                                if ((lane & 1) == 0) s_part[j - lo][hw][p] = add ? s_part[j - lo][hw][p] + h1 : h1;
                                if ((lane & 15) == 0) {
                                    s_part[j - lo][hw][8] = add ? s_part[j - lo][hw][8] + v8 : v8;
                                    atomicOr(s_wrote + (j - lo), 1u << hw);
                                }
                            }
                        }
                    }
                }
                __syncwarp();  // this region's stores and flags before the next region's reads
            }
            __syncthreads();
            // Block sum over the half-warps that wrote, in order, one record per pair.
            for (int e = threadIdx.x; e < (hi - lo) * kPart; e += G::THREADS) {
                const int j = e / kPart, c = e - j * kPart;
                const uint32_t wr = s_wrote[j];
                float s = 0.f;
#pragma unroll
                for (int w = 0; w < 2 * G::WARPS; ++w) s += ((wr >> w) & 1u) ? s_part[j][w][c] : 0.f;
                partials[(size_t)s_slot[lo + j] * kPart + c] = s;
            }
            __syncthreads();
        }
    }
};

// Tile of a frame that the backward's launch index b takes: the tile rows
// centre-out (c, c + 1, c - 1, c + 2, ..., c = (TY - 1) / 2, a bijection onto
// [0, TY) for either parity of TY), each row left to right. The rows near
// the image's centre, where the lists are longest in views of a centred
// scene, start first and the short border rows fill the end of the launch;
// neighbouring launches stay neighbouring tiles. Each tile's computation is
// the same whatever the order.
__device__ __forceinline__ int centre_out_tile(const Frame& f, int b) {
    const int r = b / f.TX, tx = b - r * f.TX;
    const int c = (f.TY - 1) / 2;
    const int ty = (r & 1) ? c + (r + 1) / 2 : c - r / 2;
    return ty * f.TX + tx;
}

// Emission slot of the pair (tile (tx, ty), Gaussian g): its first slot
// slot_of(g) plus the tile's row-major rank in g's rectangle.
template <typename SlotBase>
__device__ __forceinline__ uint32_t pair_slot(SlotBase slot_of, const uint2* __restrict__ rect, uint32_t g, int tx,
                                              int ty) {
    const uint2 rc = __ldg(rect + g);
    const uint32_t x0 = rc.x & 0xffffu, y0 = rc.x >> 16, x1 = rc.y & 0xffffu;
    return slot_of(g) + (ty - y0) * (x1 - x0 + 1) + (tx - x0);
}

// Block-wide maximum of the last-contributor counts (positions past it are
// never composited; their records are zero).
template <int TS>
__device__ __forceinline__ uint32_t block_max_last(const uint32_t* last, uint32_t* s_max, int warp, int lane) {
    using G = TileGeom<TS>;
    uint32_t my = 0;
#pragma unroll
    for (int k = 0; k < G::PPT; ++k) my = max(my, last[k]);
    for (int o = 16; o > 0; o >>= 1) my = max(my, __shfl_xor_sync(kFull, my, o));
    if (lane == 0) s_max[warp] = my;
    __syncthreads();
    uint32_t m = 0;
#pragma unroll
    for (int w = 0; w < G::WARPS; ++w) m = max(m, s_max[w]);
    return m;
}

// Zero records for list positions [from, len) that no pixel composited.
template <typename SlotBase>
__device__ __forceinline__ void zero_records(uint2 range, uint32_t from, const uint32_t* __restrict__ vals,
                                             const uint2* __restrict__ rect, SlotBase slot_of, int tx, int ty,
                                             int threads, float* __restrict__ partials) {
    const uint32_t len = range.y - range.x;
    for (uint32_t j = from + threadIdx.x; j < len; j += threads) {
        const uint32_t slot = pair_slot(slot_of, rect, __ldg(vals + range.x + j), tx, ty);
        float* dst = partials + (size_t)slot * kPart;
#pragma unroll
        for (int c = 0; c < kPart; ++c) dst[c] = 0.f;
    }
}

// Slot-ordered sum of a Gaussian's nrec pair records (kPart floats each,
// contiguous from src) into pr: the loads of four records are issued before
// their adds, and the adds keep slot order (a record past nrec adds +0, which
// leaves a sum that started at +0 bit for bit unchanged), so the result is
// that of the plain loop with a quarter of its dependent load latencies.
__device__ __forceinline__ void sum_pair_records(const float* __restrict__ src, uint32_t nrec, float (&pr)[kPart]) {
    for (uint32_t s = 0; s < nrec; s += 4) {
        float r[4][kPart];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const bool ok = s + k < nrec;
#pragma unroll
            for (int c = 0; c < kPart; ++c) r[k][c] = ok ? __ldg(src + (size_t)(s + k) * kPart + c) : 0.f;
        }
#pragma unroll
        for (int k = 0; k < 4; ++k)
#pragma unroll
            for (int c = 0; c < kPart; ++c) pr[c] += r[k][c];
    }
}

// Stages list positions [start, start + cnt) of a tile: records and masks,
// and (WITH_SLOT) each pair's emission slot. The stagings of the backward
// and of the fused training pass (WITH_SLOT) build the ellipse's sub-block
// masks, the forward's the bounding box's.
template <int TS, bool WITH_SLOT, typename Splats, typename SlotBase, int TH = TileGeom<TS>::THREADS>
__device__ __forceinline__ void stage_batch(const Frame& f, float ox, float oy, int tx, int ty, uint32_t start,
                                            int cnt, const uint32_t* __restrict__ vals, const Splats& sp,
                                            const uint2* __restrict__ rect, SlotBase slot_of, SplatRec* s_rec,
                                            typename TileGeom<TS>::Mask* s_mask, uint32_t* s_slot) {
    for (int j = threadIdx.x; j < cnt; j += TH) {
        const uint32_t g = __ldg(vals + start + j);
        typename TileGeom<TS>::Mask m;
        stage_splat<TS, WITH_SLOT>(f, ox, oy, sp, g, s_rec + rec_slot(j), m);
        s_mask[j] = m;
        if (WITH_SLOT) s_slot[j] = pair_slot(slot_of, rect, g, tx, ty);
    }
}

struct NoSlot {
    __device__ __forceinline__ uint32_t operator()(uint32_t) const { return 0u; }
};

// Forward of one tile, one thread per pixel (TS * TS threads): stages the
// list 256 splats at a time and composites each batch (FwdPixels::batch),
// then writes image = C + T bg, the final transmittance and the 1-based list
// position of the last composited splat.
template <int TS, typename Splats>
__device__ __forceinline__ void blend_tile(const Frame& f, int tile, uint2 range, const uint32_t* __restrict__ vals,
                                           const Splats& sp, float* __restrict__ image, float* __restrict__ t_final,
                                           uint32_t* __restrict__ n_contrib) {
    constexpr int TH = TS * TS;
    using G = TileGeom<TS, TH>;
    __shared__ SplatRec s_rec[rec_slots(kBlendBatch)];
    __shared__ typename G::Mask s_mask[kBlendBatch];
    const int tx = tile % f.TX, ty = tile / f.TX;
    const float ox = (float)(tx * TS), oy = (float)(ty * TS);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    init_null_splats(s_rec, kBlendBatch);
    FwdPixels<TS, TH> P;
    P.init(warp, lane);
    for (uint32_t start = range.x; start < range.y; start += kBlendBatch) {
        const int cnt = (int)min((uint32_t)kBlendBatch, range.y - start);
        __syncthreads();
        stage_batch<TS, false, Splats, NoSlot, TH>(f, ox, oy, tx, ty, start, cnt, vals, sp, nullptr, NoSlot{}, s_rec,
                                                   s_mask, nullptr);
        __syncthreads();
        P.batch(s_rec, s_mask, cnt, start + 1 - range.x, lane);
    }
#pragma unroll
    for (int k = 0; k < G::PPT; ++k) {
        const int gx = tx * TS + (int)P.px[k], gy = ty * TS + (int)P.py[k];
        if (gx < f.W && gy < f.H) {
            const size_t pix = (size_t)gy * f.W + gx;
            image[3 * pix] = fmaf(P.T[k], f.bg[0], P.C0[k]);
            image[3 * pix + 1] = fmaf(P.T[k], f.bg[1], P.C1[k]);
            image[3 * pix + 2] = fmaf(P.T[k], f.bg[2], P.C2[k]);
            t_final[pix] = P.T[k];
            n_contrib[pix] = P.last[k];
        }
    }
}

// Shared memory of the backward and fused kernels, staging BATCH splats and
// holding the partials of CHUNK of them.
template <int TS, int BATCH = kBlendBatch, int CHUNK = kBwdChunk>
struct BwdSmem {
    SplatRec rec[rec_slots(BATCH)];
    typename TileGeom<TS>::Mask mask[BATCH];
    uint32_t slot[BATCH];
    float part[CHUNK][2 * TileGeom<TS>::WARPS][kPart];
    uint32_t wrote[CHUNK];
    uint32_t maxl[TileGeom<TS>::WARPS];
};

// Shared memory of the fused training pass.
template <int TS>
using TrainSmem = BwdSmem<TS, kBlendBatch, kTrainChunk>;

// Backward of one tile from the stored forward outputs: each pair's 9
// partials at its emission slot (see BwdPixels), staging kBwdChunk splats at
// a time (the smaller shared-memory footprint keeps more blocks resident).
// `slot_of(g)` gives the first emission slot of Gaussian g's pairs for this
// frame (offsets[g] for one view, offsets[v * n + g] in a batch).
template <int TS, typename SlotBase>
__device__ __forceinline__ void blend_bwd_tile(const Frame& f, int tile, uint2 range, const uint32_t* __restrict__ vals,
                                               const float4* __restrict__ splats, const uint2* __restrict__ rect,
                                               SlotBase slot_of, const float* __restrict__ t_final,
                                               const uint32_t* __restrict__ n_contrib,
                                               const float* __restrict__ d_image, float* __restrict__ partials) {
    using G = TileGeom<TS>;
    __shared__ BwdSmem<TS, kBwdChunk> sm;
    const int tx = tile % f.TX, ty = tile / f.TX;
    const float ox = (float)(tx * TS), oy = (float)(ty * TS);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const FloatSplats sp{splats};
    BwdPixels<TS> B;
    B.init_geometry(warp, lane);
#pragma unroll
    for (int k = 0; k < G::PPT; ++k) {
        const int gx = tx * TS + (int)B.px[k], gy = ty * TS + (int)B.py[k];
        const bool inside = gx < f.W && gy < f.H;
        const size_t pix = inside ? (size_t)gy * f.W + gx : 0;
        B.T[k] = inside ? t_final[pix] : 1.f;
        B.last[k] = inside ? n_contrib[pix] : 0u;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            B.dC[k][c] = inside ? d_image[3 * pix + c] : 0.f;
            B.Bc[k][c] = f.bg[c];
        }
    }
    const uint32_t max_last = block_max_last<TS>(B.last, sm.maxl, warp, lane);
    zero_records(range, max_last, vals, rect, slot_of, tx, ty, G::THREADS, partials);
    // batches of the composited prefix [0, max_last), last batch first
    const int nb = (int)((max_last + kBwdChunk - 1) / kBwdChunk);
    for (int b = nb - 1; b >= 0; --b) {
        const uint32_t lo = (uint32_t)b * kBwdChunk;
        const int cnt = (int)min((uint32_t)kBwdChunk, max_last - lo);
        __syncthreads();
        stage_batch<TS, true>(f, ox, oy, tx, ty, range.x + lo, cnt, vals, sp, rect, slot_of, sm.rec, sm.mask,
                              sm.slot);
        __syncthreads();
        B.batch(sm.rec, sm.mask, sm.slot, sm.part, sm.wrote, cnt, lo, warp, lane, partials);
    }
}

// One training step's blend of one tile in a single pass: the forward
// composite (bit-identical to blend_tile), image and final transmittance
// written, the L2 residual d = image - target formed in registers, then the
// backward of BwdPixels over the same list. When the tile's list fits one
// batch (most tiles), the backward reuses the forward's staged records.
template <int TS, typename SlotBase>
__device__ __forceinline__ void train_tile(const Frame& f, int tile, uint2 range, const uint32_t* __restrict__ vals,
                                           const float4* __restrict__ splats, const uint2* __restrict__ rect,
                                           SlotBase slot_of, const float* __restrict__ target,
                                           float* __restrict__ image, float* __restrict__ t_final,
                                           uint32_t* __restrict__ n_contrib, float* __restrict__ partials,
                                           TrainSmem<TS>& sm) {
    using G = TileGeom<TS>;
    const int tx = tile % f.TX, ty = tile / f.TX;
    const float ox = (float)(tx * TS), oy = (float)(ty * TS);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const FloatSplats sp{splats};
    const uint32_t len = range.y - range.x;
    const int nb = (int)((len + kBlendBatch - 1) / kBlendBatch);
    init_null_splats(sm.rec, kBlendBatch);
    BwdPixels<TS, kTrainChunk> B;
    {
        FwdPixels<TS> P;
        P.init(warp, lane);
        for (int b = 0; b < nb; ++b) {
            const uint32_t lo = (uint32_t)b * kBlendBatch;
            const int cnt = (int)min((uint32_t)kBlendBatch, len - lo);
            __syncthreads();
            stage_batch<TS, true>(f, ox, oy, tx, ty, range.x + lo, cnt, vals, sp, rect, slot_of, sm.rec, sm.mask,
                                  sm.slot);
            __syncthreads();
            P.batch(sm.rec, sm.mask, cnt, lo + 1, lane);
        }
        B.init_geometry(warp, lane);
#pragma unroll
        for (int k = 0; k < G::PPT; ++k) {
            const int gx = tx * TS + (int)P.px[k], gy = ty * TS + (int)P.py[k];
            const bool inside = gx < f.W && gy < f.H;
            const size_t pix = inside ? (size_t)gy * f.W + gx : 0;
            const float img[3] = {fmaf(P.T[k], f.bg[0], P.C0[k]), fmaf(P.T[k], f.bg[1], P.C1[k]),
                                  fmaf(P.T[k], f.bg[2], P.C2[k])};
            if (inside) {
                image[3 * pix] = img[0];
                image[3 * pix + 1] = img[1];
                image[3 * pix + 2] = img[2];
                t_final[pix] = P.T[k];
                n_contrib[pix] = P.last[k];
            }
            B.T[k] = inside ? P.T[k] : 1.f;
            B.last[k] = inside ? P.last[k] : 0u;
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                B.dC[k][c] = inside ? img[c] - __ldg(target + 3 * pix + c) : 0.f;
                B.Bc[k][c] = f.bg[c];
            }
        }
    }
    const uint32_t max_last = block_max_last<TS>(B.last, sm.maxl, warp, lane);
    zero_records(range, max_last, vals, rect, slot_of, tx, ty, G::THREADS, partials);
    const int nbb = (int)((max_last + kBlendBatch - 1) / kBlendBatch);
    for (int b = nbb - 1; b >= 0; --b) {
        const uint32_t lo = (uint32_t)b * kBlendBatch;
        const int cnt = (int)min((uint32_t)kBlendBatch, max_last - lo);
        if (b != nb - 1) {  // the last forward batch is still staged
            __syncthreads();
            stage_batch<TS, true>(f, ox, oy, tx, ty, range.x + lo, cnt, vals, sp, rect, slot_of, sm.rec, sm.mask,
                                  sm.slot);
        }
        __syncthreads();
        B.batch(sm.rec, sm.mask, sm.slot, sm.part, sm.wrote, cnt, lo, warp, lane, partials);
    }
}

}  // namespace ws
