// Rasterisation stage (paper §3.4 with the compositing of §2.1), re-designed
// as a per-tile CUDA blend: one block per screen tile, one thread per pixel,
// front to back over the tile's depth-sorted pair list.
//
// Per pair:  a = min(0.99, sigma exp(-q/2)), q = d^T conic d, d = pixel
// centre - splat centre; a < 1/255 is skipped; C += c a T; T *= 1 - a.
//
// The splats of a tile are staged through shared memory in batches of 256:
// each thread gathers one splat record (value -> Gaussian index -> its
// 48-byte record: centre, conic, opacity, colour), converts its centre to
// tile-relative coordinates with the double-float centre (so pixel offsets
// carry no large-magnitude rounding), folds -log2(e)/2 into the conic so the
// exponent is one ex2 instruction, and computes the box of its
// opacity-aware extent (§3.4). A half-warp covers a 4x4 pixel sub-block; a
// splat whose box misses the sub-block is skipped by that half-warp, which
// removes most of the evaluations of small splats that only graze a tile.
//
// FP32-pipe + SFU bound: ~17 FP32 instructions and one ex2 per evaluated
// (pixel, splat) pair.
#include "ws_blend.cuh"
#include "ws_common.cuh"
#include "ws_kernels.cuh"

namespace ws {

namespace {

constexpr int kRangeThreads = 256;

// ranges[t] = [start, end) of tile t in the sorted key list, for every tile
// (an empty tile gets start = end), in one pass over positions 0..n: at
// position i, between the tiles a of key i-1 and c of key i, tiles a+1..c
// start and tiles a..c-1 end (scan_boundaries). Keys whose tile is >= ntiles
// (none in a frame) count as past the end.
__global__ void __launch_bounds__(kRangeThreads)
k_tile_ranges(const uint64_t* __restrict__ keys, const uint32_t* __restrict__ num_keys,
              uint2* __restrict__ ranges, uint32_t ntiles) {
    pdl_wait();
    const int lane = threadIdx.x & 31;
    const int64_t nt = (int64_t)ntiles;
    scan_boundaries<4>(
        keys, *num_keys, nt, [nt](uint64_t k) { return min((int64_t)(k >> 31), nt); },
        [&](int64_t lo, int64_t hi, uint32_t pos) {
            for (int64_t t = lo + lane; t <= hi; t += kWarp) {
                if (t >= 0 && t < hi && t < nt) ranges[t].y = pos;
                if (t > lo && t < nt) ranges[t].x = pos;
            }
        });
}

template <int TS>
__global__ void __launch_bounds__(TS * TS, blend_min_blocks<TS>())
k_blend(const uint2* __restrict__ ranges, const uint32_t* __restrict__ vals, const float4* __restrict__ splats,
        const Frame f, float* __restrict__ image, float* __restrict__ t_final, uint32_t* __restrict__ n_contrib) {
    pdl_wait();
    const FloatSplats sp{splats};
    blend_tile<TS>(f, blockIdx.x, ranges[blockIdx.x], vals, sp, image, t_final, n_contrib);
}

}  // namespace

cudaError_t launch_tile_ranges(const uint64_t* keys, const uint32_t* num_keys, uint32_t* ranges, uint32_t ntiles,
                               uint32_t flags, cudaStream_t stream) {
    if (flags & WS_CFG_RANGES_GIVEN) return cudaSuccess;
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    uint2* r2w = reinterpret_cast<uint2*>(ranges);
    return launch_pdl(k_tile_ranges, dim3(sms * 8), dim3(kRangeThreads), 0, stream, keys, num_keys, r2w, ntiles);
}

cudaError_t launch_rasterize(const uint32_t* num_keys, int64_t /*key_capacity_hint*/,
                             const uint64_t* keys, const uint32_t* vals, const float* splats,
                             const Frame& f, uint32_t* ranges, float* image, float* t_final,
                             uint32_t* n_contrib, cudaStream_t stream) {
    const int ntiles = f.TX * f.TY;
    if (ntiles == 0) return cudaSuccess;
    cudaError_t e = launch_tile_ranges(keys, num_keys, ranges, (uint32_t)ntiles, f.flags, stream);
    if (e != cudaSuccess) return e;
    const uint2* r2 = reinterpret_cast<const uint2*>(ranges);
    const float4* s4 = reinterpret_cast<const float4*>(splats);
    switch (f.TS) {
        case 8:
            return launch_pdl(k_blend<8>, dim3(ntiles), dim3(64), 0, stream, r2, vals, s4, f, image, t_final,
                              n_contrib);
        case 16:
            return launch_pdl(k_blend<16>, dim3(ntiles), dim3(256), 0, stream, r2, vals, s4, f, image, t_final,
                              n_contrib);
        case 32:
            return launch_pdl(k_blend<32>, dim3(ntiles), dim3(1024), 0, stream, r2, vals, s4, f, image, t_final,
                              n_contrib);
        default:
            return cudaErrorInvalidValue;
    }
}

}  // namespace ws
