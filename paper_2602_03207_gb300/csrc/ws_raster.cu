// Rasterisation stage (paper §3.4 with the compositing of §2.1), re-designed
// as a per-tile CUDA blend: one block per screen tile, one thread per pixel,
// front to back over the tile's depth-sorted pair list.
//
// Per pair:  a = min(0.99, sigma exp(-q/2)), q = d^T conic d, d = pixel
// centre - splat centre; a < 1/255 is skipped; C += c a T; T *= 1 - a.
//
// The splats of a tile are staged through shared memory in batches of 256:
// each thread gathers one splat (value -> Gaussian index -> centre, conic,
// opacity, colour), converts its centre to tile-relative coordinates with
// the double-float centre (so pixel offsets carry no large-magnitude
// rounding), folds -log2(e)/2 into the conic so the exponent is one ex2
// instruction, and computes the box of its opacity-aware extent (§3.4).
// A warp covers an 8x4 pixel block; a splat whose box misses the block is
// skipped by the whole warp at once (a warp-uniform branch), which removes
// most of the evaluations of small splats that only graze a tile.
//
// FP32-pipe + SFU bound: ~17 FP32 instructions and one ex2 per evaluated
// (pixel, splat) pair.
#include "ws_common.cuh"
#include "ws_kernels.cuh"

namespace ws {

namespace {

constexpr int kRangeThreads = 256;

// ranges[t] = [start, end) of tile t in the sorted key list. Tiles with no
// pairs keep the zero range from the preceding memset. Grid-stride over the
// device-side key count.
__global__ void __launch_bounds__(kRangeThreads)
k_tile_ranges(const uint64_t* __restrict__ keys, const uint32_t* __restrict__ num_keys,
              uint2* __restrict__ ranges, uint32_t ntiles) {
    const uint32_t n = *num_keys;
    for (uint32_t p = blockIdx.x * kRangeThreads + threadIdx.x; p < n; p += gridDim.x * kRangeThreads) {
        uint32_t t = (uint32_t)(__ldg(keys + p) >> 31);
        uint32_t prev = p > 0 ? (uint32_t)(__ldg(keys + p - 1) >> 31) : 0xffffffffu;
        uint32_t next = p + 1 < n ? (uint32_t)(__ldg(keys + p + 1) >> 31) : 0xffffffffu;
        if (t >= ntiles) continue;  // not a key of this tile grid
        if (t != prev) ranges[t].x = p;
        if (t != next) ranges[t].y = p + 1;
    }
}

constexpr int kBlendBatch = 256;

// Shared-memory record of one splat for the blend (48 bytes).
struct SplatRec {
    float4 geo;   // tile-relative centre x, y; conic premultiplied A, B
    float4 geo2;  // C, opacity, -, -
    float4 col;   // r, g, b, -
};

// One block per tile. Each warp owns WPB (TS^2/256, at least 1) 8x4 pixel
// blocks. Splats are staged 256 at a time; while staging, every splat also
// records the bitmask of the tile's 8x4 blocks that its opacity-aware
// extent box reaches. Each warp then walks the batch 32 splats at a time,
// ballots the bit of its own block and visits only those splats, in list
// order, so per pixel the compositing order is unchanged.
template <int TS>
__global__ void __launch_bounds__(TS * TS >= 256 ? 256 : TS * TS)
k_blend(const uint2* __restrict__ ranges, const uint32_t* __restrict__ vals,
        const float4* __restrict__ mean2d, const float* __restrict__ conic,
        const float* __restrict__ opacity, const float* __restrict__ rgb, const Frame f,
        float* __restrict__ image, float* __restrict__ t_final, uint32_t* __restrict__ n_contrib) {
    constexpr int THREADS = TS * TS >= 256 ? 256 : TS * TS;
    constexpr int WARPS = THREADS / 32;
    constexpr int PPT = TS * TS / THREADS;  // pixel blocks per warp (TS = 32: 4)
    constexpr int BW = 8, BH = 4;           // warp pixel block
    constexpr int BPR = TS / BW;            // blocks per row
    constexpr int BROWS = TS / BH;          // block rows
    static_assert(BPR * BROWS <= 32, "block mask is 32 bits");
    __shared__ SplatRec s_rec[kBlendBatch];
    __shared__ uint32_t s_mask[kBlendBatch];

    const int tile = blockIdx.x;
    const int tx = tile % f.TX, ty = tile / f.TX;
    const float ox = (float)(tx * TS), oy = (float)(ty * TS);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint2 range = ranges[tile];

    float px[PPT], py[PPT], T[PPT], C0[PPT], C1[PPT], C2[PPT];
    uint32_t last[PPT];
#pragma unroll
    for (int k = 0; k < PPT; ++k) {
        const int b = warp + k * WARPS;
        const int bx = (b % BPR) * BW, by = (b / BPR) * BH;
        px[k] = (float)(bx + (lane & 7)) + 0.5f;
        py[k] = (float)(by + (lane >> 3)) + 0.5f;
        T[k] = 1.f;
        C0[k] = C1[k] = C2[k] = 0.f;
        last[k] = 0;
    }

    for (uint32_t start = range.x; start < range.y; start += kBlendBatch) {
        const int cnt = (int)min((uint32_t)kBlendBatch, range.y - start);
        __syncthreads();
        for (int j = threadIdx.x; j < cnt; j += THREADS) {
            const uint32_t g = __ldg(vals + start + j);
            const float4 m = __ldg(mean2d + g);
            const float a = __ldg(conic + 3 * g), b = __ldg(conic + 3 * g + 1), c = __ldg(conic + 3 * g + 2);
            const float op = __ldg(opacity + g);
            SplatRec r;
            r.geo.x = __fadd_rn(__fsub_rn(m.x, ox), m.z);
            r.geo.y = __fadd_rn(__fsub_rn(m.y, oy), m.w);
            r.geo.z = -0.5f * kLog2e * a;
            r.geo.w = -kLog2e * b;
            r.geo2 = make_float4(-0.5f * kLog2e * c, op, 0.f, 0.f);
            r.col = make_float4(__ldg(rgb + 3 * g), __ldg(rgb + 3 * g + 1), __ldg(rgb + 3 * g + 2), 0.f);
            s_rec[j] = r;
            // Box of the ellipse where the alpha reaches 1/255 (§3.4), with a
            // small margin so rounding never drops a pair the per-pixel test
            // would keep: half-widths sqrt(q_c Sigma'_xx), sqrt(q_c Sigma'_yy).
            const float det = fmaf(a, c, -b * b);
            const float qc = fmaxf(0.f, 2.f * (kLn255 + __logf(op)));
            const float ex = sqrtf(qc * c / det) * 1.0001f + 1e-3f;
            const float ey = sqrtf(qc * a / det) * 1.0001f + 1e-3f;
            // blocks whose pixel centres [8c + .5, 8c + 7.5] x [4r + .5, 4r + 3.5] meet the box
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
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < PPT; ++k) {
            const int blk = warp + k * WARPS;
            for (int base = 0; base < cnt; base += 32) {
                const int jj = base + lane;
                uint32_t bits = __ballot_sync(kFull, jj < cnt && ((s_mask[jj] >> blk) & 1u));
                while (bits) {
                    const int j = base + __ffs(bits) - 1;
                    bits &= bits - 1;
                    const float4 geo = s_rec[j].geo;
                    const float4 geo2 = s_rec[j].geo2;
                    const float dx = px[k] - geo.x, dy = py[k] - geo.y;
                    const float alpha = splat_alpha(dx, dy, geo.z, geo.w, geo2.x, geo2.y);
                    if (alpha < kAlphaMin) continue;
                    const float4 col = s_rec[j].col;
                    const float w = alpha * T[k];
                    C0[k] = fmaf(col.x, w, C0[k]);
                    C1[k] = fmaf(col.y, w, C1[k]);
                    C2[k] = fmaf(col.z, w, C2[k]);
                    T[k] = T[k] - w;
                    last[k] = start + j + 1 - range.x;
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

}  // namespace

cudaError_t launch_rasterize(const uint32_t* num_keys, int64_t /*key_capacity_hint*/,
                             const uint64_t* keys, const uint32_t* vals, const float* mean2d,
                             const float* conic, const float* opacity, const float* rgb,
                             const Frame& f, uint32_t* ranges, float* image, float* t_final,
                             uint32_t* n_contrib, cudaStream_t stream) {
    const int ntiles = f.TX * f.TY;
    if (ntiles == 0) return cudaSuccess;
    cudaError_t e = cudaMemsetAsync(ranges, 0, (size_t)ntiles * 2 * sizeof(uint32_t), stream);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    k_tile_ranges<<<sms * 4, kRangeThreads, 0, stream>>>(keys, num_keys, reinterpret_cast<uint2*>(ranges),
                                                     (uint32_t)ntiles);
    const uint2* r2 = reinterpret_cast<const uint2*>(ranges);
    const float4* m4 = reinterpret_cast<const float4*>(mean2d);
    switch (f.TS) {
        case 8:
            k_blend<8><<<ntiles, 64, 0, stream>>>(r2, vals, m4, conic, opacity, rgb, f, image, t_final, n_contrib);
            break;
        case 16:
            k_blend<16><<<ntiles, 256, 0, stream>>>(r2, vals, m4, conic, opacity, rgb, f, image, t_final, n_contrib);
            break;
        case 32:
            k_blend<32><<<ntiles, 256, 0, stream>>>(r2, vals, m4, conic, opacity, rgb, f, image, t_final, n_contrib);
            break;
        default:
            return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace ws
