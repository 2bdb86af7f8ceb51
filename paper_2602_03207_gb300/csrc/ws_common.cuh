// Device helpers shared by the render-path kernels (sm_103a).
#pragma once

#include <cstdint>
#include <utility>
#include <cuda_runtime.h>

#include "websplat.h"

namespace ws {

constexpr int kWarp = 32;
constexpr uint32_t kFull = 0xffffffffu;

// Bytes reserved at the head of every workspace for the status words.
constexpr size_t kStatusBytes = 256;

// Per-Gaussian splat record written by the pre-processing and read by the
// blends (three float4: centre (x_hi, y_hi, x_lo, y_lo); conic a, b, c and
// opacity sigma; colour r, g, b and a zero), so a gather of one splat touches
// two 32-byte sectors instead of one per separate array.
constexpr int kSplatFloats = 12;
constexpr int kSplatVec4 = kSplatFloats / 4;

// Camera and frame constants, derived on the host once per call and passed
// by value to every kernel.
struct Frame {
    float R[9];       // world -> camera rotation, row-major
    float t[3];       // world -> camera translation
    float campos[3];  // camera centre in world coordinates (-R^T t)
    float fx, fy, cx, cy;
    float znear;
    float limx, limy; // guard-band limits of t_x/t_z and t_y/t_z inside J
    float dilation;
    float bg[3];
    int W, H;
    int TS, TX, TY;   // tile side and tile grid
    uint32_t flags;
};

// Several cameras of one scene rendered as one batch (at most kMaxViews).
// Per-(view, Gaussian) arrays are view-major: element (v, g) is at v * n + g.
// View v's tiles are numbered tile_off[v] .. tile_off[v+1]-1 in one global
// tile grid and its pixels start at pix_off[v] in the packed image.
constexpr int kMaxViews = 64;

struct ViewGrid {
    uint32_t tiles_x[kMaxViews];
    uint32_t tile_off[kMaxViews + 1];
    int views;
};

struct FrameTable {
    Frame f[kMaxViews];
    uint32_t tile_off[kMaxViews + 1];
    uint64_t pix_off[kMaxViews + 1];
    int views;
};

// The view owning global tile t (binary search over tile_off).
__device__ __forceinline__ int view_of_tile(const uint32_t* tile_off, int views, uint32_t t) {
    int lo = 0, hi = views - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (tile_off[mid] <= t) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// ---------------------------------------------------------------------------
// Double-float ("unevaluated sum of two floats") arithmetic. Error-free
// transformations of Knuth (two-sum) and Dekker (two-product via a fused
// multiply-add); intrinsics keep the compiler from contracting or
// reassociating them.
struct DF {
    float hi, lo;
};

__device__ __forceinline__ DF two_sum(float a, float b) {
    float s = __fadd_rn(a, b);
    float bb = __fsub_rn(s, a);
    float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return {s, e};
}

__device__ __forceinline__ DF quick_two_sum(float a, float b) {  // |a| >= |b|
    float s = __fadd_rn(a, b);
    float e = __fsub_rn(b, __fsub_rn(s, a));
    return {s, e};
}

__device__ __forceinline__ DF two_prod(float a, float b) {
    float p = __fmul_rn(a, b);
    float e = __fmaf_rn(a, b, -p);
    return {p, e};
}

// r0*x + r1*y + r2*z + t in double-float (inputs exact floats).
__device__ __forceinline__ DF df_affine3(float r0, float r1, float r2, float x, float y, float z,
                                         float t) {
    DF acc = {t, 0.f};
    DF p = two_prod(r0, x);
    DF s = two_sum(acc.hi, p.hi);
    float lo = __fadd_rn(p.lo, s.lo);
    acc.hi = s.hi;
    p = two_prod(r1, y);
    s = two_sum(acc.hi, p.hi);
    lo = __fadd_rn(lo, __fadd_rn(p.lo, s.lo));
    acc.hi = s.hi;
    p = two_prod(r2, z);
    s = two_sum(acc.hi, p.hi);
    lo = __fadd_rn(lo, __fadd_rn(p.lo, s.lo));
    return quick_two_sum(s.hi, lo);
}

// a / b for double-float a, b (one Newton-style correction step).
__device__ __forceinline__ DF df_div(DF a, DF b) {
    float q1 = __fdiv_rn(a.hi, b.hi);
    DF p = two_prod(q1, b.hi);
    float r = __fsub_rn(__fsub_rn(a.hi, p.hi), p.lo);
    r = __fadd_rn(r, a.lo);
    r = __fsub_rn(r, __fmul_rn(q1, b.lo));
    float q2 = __fdiv_rn(r, b.hi);
    return quick_two_sum(q1, q2);
}

// f * u + c for float f, c and double-float u.
__device__ __forceinline__ DF df_scale_add(float f, DF u, float c) {
    DF p = two_prod(f, u.hi);
    float plo = __fmaf_rn(f, u.lo, p.lo);
    DF s = two_sum(p.hi, c);
    return quick_two_sum(s.hi, __fadd_rn(s.lo, plo));
}

// ---------------------------------------------------------------------------
// 2^x on the special-function unit (the PTX ex2.approx instruction).
__device__ __forceinline__ float ex2_approx(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// log2(x) on the special-function unit (PTX lg2.approx: absolute error about
// 2^-22). The blends take L = log2(sigma) from it, forward and backward alike.
__device__ __forceinline__ float lg2_approx(float x) {
    float y;
    asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// 1/x and sqrt(x) on the special-function unit (PTX rcp.approx, sqrt.approx:
// a few ulp). Used only where a margin absorbs the error (block masks).
__device__ __forceinline__ float rcp_approx(float x) {
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float sqrt_approx(float x) {
    float y;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

constexpr float kLog2e = 1.4426950408889634f;
constexpr float kAlphaMin = 1.0f / 255.0f;  // §3.4 quantisation threshold
constexpr float kAlphaMax = 0.99f;
// ln(255): the extent threshold is q_c = 2 (ln 255 + ln sigma).
constexpr float kLn255 = 5.541263545158426f;
// sigma < 1/255  <=>  logit < -ln(254)
constexpr double kOpacityLogitMin = -5.537334267018537;

// log2 of the unclamped splat alpha sigma exp(-q/2) at offset (dx, dy) from
// the centre, with the conic premultiplied (A = -log2(e) a / 2, B = -log2(e) b,
// C = -log2(e) c / 2) and L = log2(sigma):
//     e = A dx^2 + B dx dy + C dy^2 + L.
// A pair is composited iff e >= log2(1/255) (alpha >= 1/255, §3.4's
// threshold), and then alpha = min(0.99, 2^e). The forward and the backward
// blend both decide and evaluate through this function, so they agree on
// every pair.
constexpr float kLog2AlphaMin = -7.994353436858858f;  // log2(1/255)
constexpr float kTwoLn2 = 1.3862943611198906f;
constexpr float kLn2 = 0.6931471805599453f;
// The extent threshold from L = log2(sigma): e >= log2(1/255) <=> q <= q_c
// with q_c = 2 ln 2 (L - log2(1/255)) = 2 (ln 255 + ln sigma).

__device__ __forceinline__ float splat_log2_alpha(float dx, float dy, float A, float B, float C, float L) {
    const float u = __fmaf_rn(A, dx, __fmul_rn(B, dy));
    return __fmaf_rn(dx, u, __fmaf_rn(__fmul_rn(C, dy), dy, L));
}

// The splat's axis basis from t = tan(theta / 2): e1 = (ct, st) along the
// major axis of Sigma', e2 = (-st, ct). The pre-processing stores t, and
// the backward blend and the pre-processing adjoint both rebuild the basis
// here, so they use the same one to the last bit.
__device__ __forceinline__ void axis_basis(float t, float& ct, float& st) {
    const float r = rcp_approx(fmaf(t, t, 1.f));  // |e1| = 1 to a few ulp
    ct = fmaf(-t, t, 1.f) * r;
    st = 2.f * t * r;
}


// ---------------------------------------------------------------------------
// Block-wide exclusive scan of one uint32 per thread (THREADS threads).
// `smem` must hold THREADS / 32 + 1 words. Returns the exclusive prefix and
// writes the block total to *total.
template <int THREADS>
__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t v, uint32_t* smem,
                                                         uint32_t* total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(kFull, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) smem[warp] = x;
    __syncthreads();
    if (warp == 0) {
        constexpr int NW = THREADS / 32;
        uint32_t w = lane < NW ? smem[lane] : 0u;
        uint32_t s = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(kFull, s, o);
            if (lane >= o) s += y;
        }
        if (lane < NW) smem[lane] = s - w;
        if (lane == NW - 1) smem[NW] = s;
    }
    __syncthreads();
    uint32_t r = smem[warp] + x - v;
    *total = smem[THREADS / 32];
    __syncthreads();
    return r;
}

// ---------------------------------------------------------------------------
// Programmatic dependent launch. Every kernel of the path is launched with
// programmatic stream serialisation and calls pdl_wait() before its first
// global-memory access (read or write), which returns once the predecessor
// grid has completed and its writes are visible. No kernel triggers its
// dependents early (griddepcontrol.launch_dependents): a successor launches
// as its predecessor's blocks exit, with the launch itself already prepared,
// which measured faster than an early trigger (whose waiting blocks occupy
// the SMs) and than no programmatic launch. Ordering and results are those
// of plain stream order.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

template <typename... KArgs, typename... Args>
cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t stream,
                       Args&&... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

// Bitmask of a tile's BW x BH pixel blocks (BPR per row, BROWS rows, bit
// row * BPR + col) whose pixel centres [BW col + .5, BW col + BW - .5] x
// [BH row + .5, BH row + BH - .5] meet the box [xl, xh] x [yl, yh]
// (tile-relative): one compare pair per block column and per block row.
template <int BW, int BH, int BPR, int BROWS>
__device__ __forceinline__ uint32_t box_block_mask(float xl, float xh, float yl, float yh) {
    static_assert(BPR * BROWS <= 32, "block mask is 32 bits");
    uint32_t cols = 0;
#pragma unroll
    for (int c = 0; c < BPR; ++c)
        cols |= (xl <= (float)(c * BW) + (BW - 0.5f) && xh >= (float)(c * BW) + 0.5f) ? (1u << c) : 0u;
    uint32_t mask = 0;
#pragma unroll
    for (int r = 0; r < BROWS; ++r)
        mask |= (yl <= (float)(r * BH) + (BH - 0.5f) && yh >= (float)(r * BH) + 0.5f) ? (cols << (r * BPR)) : 0u;
    return mask;
}

// Segment boundaries of a sorted key list of n keys, warp-cooperatively over
// a grid-stride loop. The segment id of position i is seg_of(keys[i]) for
// i < n, -1 before the list and end_id at i = n (ids are non-decreasing).
// For every position i in [0, n] whose id c exceeds the previous position's
// id a, the whole warp calls fill(a, c, i) and shares the ids a..c among its
// lanes, so a long run of empty segments does not serialise one thread. Each
// lane issues U independent key loads before using any of them.
template <int U, typename SegOf, typename Fill>
__device__ __forceinline__ void scan_boundaries(const uint64_t* __restrict__ keys, uint32_t n, int64_t end_id,
                                                SegOf seg_of, Fill fill) {
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    constexpr int64_t kSpan = (int64_t)kWarp * U;
    for (int64_t w = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); w * kSpan <= (int64_t)n;
         w += warps) {
        const int64_t base = w * kSpan;
        int64_t id[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int64_t i = base + u * kWarp + lane;
            id[u] = i < (int64_t)n ? seg_of(__ldg(keys + i)) : end_id;
        }
        int64_t prev = base == 0 ? -1 : seg_of(__ldg(keys + base - 1));
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int64_t i = base + u * kWarp + lane;
            const int64_t c = id[u];
            int64_t a = __shfl_up_sync(kFull, c, 1);
            if (lane == 0) a = prev;
            prev = __shfl_sync(kFull, c, 31);
            uint32_t todo = __ballot_sync(kFull, i <= (int64_t)n && c > a);
            while (todo) {
                const int src = __ffs(todo) - 1;
                todo &= todo - 1;
                fill(__shfl_sync(kFull, a, src), __shfl_sync(kFull, c, src),
                     (uint32_t)__shfl_sync(kFull, (uint32_t)i, src));
            }
        }
    }
}

__device__ __forceinline__ uint32_t lanemask_lt() {
    uint32_t m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// Lanes of the warp holding the same BITS-bit digit as this lane: one ballot
// per bit (inverted where this lane's bit is 0), ANDed together. Its cost does
// not depend on how many distinct digits the warp holds. Lanes passing
// `valid` = false take part in the votes but match no valid lane.
template <int BITS>
__device__ __forceinline__ uint32_t warp_match_digit(uint32_t digit, bool valid) {
    uint32_t peers = __ballot_sync(kFull, valid);
    if (!valid) peers = ~peers;
#pragma unroll
    for (int b = 0; b < BITS; ++b) {
        const bool bit = (digit >> b) & 1u;
        const uint32_t vote = __ballot_sync(kFull, bit);
        peers &= bit ? vote : ~vote;
    }
    return peers;
}

__device__ __forceinline__ void set_flag(uint32_t* status, uint32_t bit) {
    // A plain store of a fixed value: every writer stores the same bit to
    // its own word, so no read-modify-write is needed.
    status[bit == WS_FLAG_CAPACITY ? 0 : 1] = 1u;
}

}  // namespace ws
