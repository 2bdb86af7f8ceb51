// Optional single-sweep variant of the radix sort (ws_config flag
// WS_CFG_SORT_LOOKBACK): the same stable LSD sort and the same result as the
// wait-free three-dispatch passes of ws_sort.cu, with the per-pass histogram
// and scan folded into one kernel by decoupled look-back.
//
//   k_lb_hist       one read of the keys: digit counts of EVERY pass (a
//                   digit's count does not depend on the order the earlier
//                   passes leave), per-block partials in shared memory.
//   k_lb_hist_scan  per pass: fixed-order sum of the partials and an
//                   exclusive scan over digits -> base_d.
//   k_lb_pass       one kernel per pass over a persistent grid: each tile
//                   ranks its keys (as the downsweep does), publishes its
//                   per-digit counts, sums its predecessors' counts by
//                   looking back until an inclusive prefix is found
//                   (prefix_wg), publishes its own inclusive prefix, then
//                   scatters to base_d + prefix_wg + local position.
//
// The published words are (state << 32 | count), written with release
// stores and read with acquire loads (no read-modify-write atomics). The
// prefixes a tile obtains are exact sums, so the result is identical under
// any scheduling; only progress depends on scheduling. Progress holds
// because every tile waits only on lower tiles, each block takes its tiles in
// increasing order and the grid is sized to be co-resident. Every wait is
// bounded (about a second): on expiry the kernel raises WS_FLAG_TIMEOUT in
// the workspace status word, every other waiter stops, tiles that could not
// complete their look-back write nothing, and the launch returns.
//
// The status words alternate between two buffers: pass p uses one and
// clears the other for pass p + 1, so no stale flag survives into the next
// pass or the next graph replay.
#include <atomic>

#include "ws_common.cuh"
#include "ws_kernels.cuh"

namespace ws {

namespace {

constexpr int kLbThreads = 256;
constexpr int kLbWarps = kLbThreads / kWarp;
constexpr int kLbItems = 8;
constexpr int kLbTile = kLbThreads * kLbItems;
constexpr int kLbHistBlocks = 512;
constexpr int kLbMaxPasses = 16;
constexpr int kLbMaxBits = 9;
constexpr uint64_t kStateAgg = 1, kStateIncl = 2;
constexpr uint32_t kMaxSpin = 1u << 22;  // x ~256 ns of sleep: about one second

__device__ __forceinline__ void st_release(uint64_t* p, uint64_t v) {
    asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__device__ __forceinline__ uint64_t ld_acquire(const uint64_t* p) {
    uint64_t v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ uint32_t ld_volatile(const uint32_t* p) {
    return *reinterpret_cast<const volatile uint32_t*>(p);
}

template <int BITS>
__global__ void __launch_bounds__(kLbThreads)
k_lb_hist(const uint64_t* __restrict__ keys, const uint32_t* __restrict__ num_keys, int begin_bit, int passes,
          int end_bit, uint32_t* __restrict__ partials, uint64_t* __restrict__ status0, int64_t status_words,
          uint32_t* __restrict__ flags, uint32_t cap) {
    constexpr int R = 1 << BITS;
    extern __shared__ __align__(16) uint32_t s_h[];  // [passes][R]
    for (int e = threadIdx.x; e < passes * R; e += kLbThreads) s_h[e] = 0;
    pdl_wait();
    if (blockIdx.x == 0 && threadIdx.x == 0) flags[1] = 0u;  // this sort's timeout word
    const int64_t gstride = (int64_t)gridDim.x * kLbThreads;
    for (int64_t e = (int64_t)blockIdx.x * kLbThreads + threadIdx.x; e < status_words; e += gstride) status0[e] = 0;
    __syncthreads();
    const uint32_t n = min(*num_keys, cap);
    const int lane = threadIdx.x & 31;
    for (int64_t base = (int64_t)blockIdx.x * kLbThreads; base < n; base += gstride) {
        const int64_t i = base + threadIdx.x;
        const bool ok = i < n;
        const uint64_t k = ok ? __ldg(keys + i) : 0ull;
        for (int p = 0; p < passes; ++p) {
            const int shift = begin_bit + p * BITS;
            const int bits = end_bit - shift < BITS ? end_bit - shift : BITS;
            const uint32_t d = (uint32_t)(k >> shift) & ((1u << bits) - 1u);
            const uint32_t peers = warp_match_digit<BITS>(d, ok);
            if (ok && lane == __ffs(peers) - 1) atomicAdd(&s_h[p * R + d], (uint32_t)__popc(peers));
        }
    }
    __syncthreads();
    uint32_t* dst = partials + (size_t)blockIdx.x * passes * R;
    for (int e = threadIdx.x; e < passes * R; e += kLbThreads) dst[e] = s_h[e];
}

// One block per pass: total of each digit over the partials in block order,
// then an exclusive scan over digits.
template <int BITS>
__global__ void __launch_bounds__(1 << BITS > 256 ? 1 << BITS : 256)
k_lb_hist_scan(const uint32_t* __restrict__ partials, int passes, uint32_t* __restrict__ base) {
    constexpr int R = 1 << BITS;
    constexpr int T = R > 256 ? R : 256;
    __shared__ uint32_t s_red[T / 32 + 1];
    pdl_wait();
    const int p = blockIdx.x, d = threadIdx.x;
    uint32_t tot = 0;
    if (d < R)
        for (int b = 0; b < kLbHistBlocks; ++b) tot += __ldg(partials + ((size_t)b * passes + p) * R + d);
    uint32_t total;
    const uint32_t ex = block_exclusive_scan<T>(tot, s_red, &total);
    if (d < R) base[p * R + d] = ex;
}

template <int BITS>
__global__ void __launch_bounds__(kLbThreads)
k_lb_pass(const uint64_t* __restrict__ keys_in, const uint32_t* __restrict__ vals_in,
          uint64_t* __restrict__ keys_out, uint32_t* __restrict__ vals_out, const uint32_t* __restrict__ num_keys,
          int shift, uint32_t mask, const uint32_t* __restrict__ base, uint64_t* __restrict__ st_cur,
          uint64_t* __restrict__ st_next, uint32_t* __restrict__ flags, int drop_tile, uint32_t cap) {
    constexpr int R = 1 << BITS;
    constexpr int kPer = R > kLbThreads ? R / kLbThreads : 1;
    extern __shared__ __align__(16) unsigned char s_raw[];
    uint64_t* s_keys = reinterpret_cast<uint64_t*>(s_raw);
    uint32_t* s_vals = reinterpret_cast<uint32_t*>(s_keys + kLbTile);
    auto s_wh = reinterpret_cast<uint16_t (*)[R]>(s_vals + kLbTile);
    uint32_t* s_start = reinterpret_cast<uint32_t*>(&s_wh[kLbWarps][0]);
    uint32_t* s_goff = s_start + R;
    uint32_t* s_red = s_goff + R;
    __shared__ int s_ok;

    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    pdl_wait();
    const uint32_t n = min(*num_keys, cap);
    const int tiles = (int)((n + kLbTile - 1) / kLbTile);
    const uint32_t lt = lanemask_lt();
    for (int tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
        for (int d = threadIdx.x; d < kLbWarps * R; d += kLbThreads) (&s_wh[0][0])[d] = 0;
        if (threadIdx.x == 0) s_ok = 1;
        __syncthreads();
        const int64_t tile_base = (int64_t)tile * kLbTile;
        const int count = (int)(((int64_t)n - tile_base) < kLbTile ? ((int64_t)n - tile_base) : kLbTile);
        const int64_t wbase = tile_base + warp * (kWarp * kLbItems);
        uint64_t key[kLbItems];
        uint32_t val[kLbItems], dig[kLbItems];
        uint16_t rnk[kLbItems];
#pragma unroll
        for (int k = 0; k < kLbItems; ++k) {
            const int64_t idx = wbase + k * kWarp + lane;
            const bool ok = idx < (int64_t)n;
            key[k] = ok ? __ldg(keys_in + idx) : 0ull;
            val[k] = ok ? __ldg(vals_in + idx) : 0u;
            dig[k] = ok ? (uint32_t)(key[k] >> shift) & mask : (uint32_t)R;
        }
#pragma unroll
        for (int k = 0; k < kLbItems; ++k) {
            const uint32_t d = dig[k];
            const bool ok = d < (uint32_t)R;
            const uint32_t peers = warp_match_digit<BITS>(d, ok);
            const int leader = __ffs(peers) - 1;
            uint32_t prior = 0;
            if (lane == leader && ok) prior = s_wh[warp][d];
            prior = __shfl_sync(kFull, prior, leader);
            rnk[k] = (uint16_t)(prior + __popc(peers & lt));
            if (lane == leader && ok) s_wh[warp][d] = (uint16_t)(prior + __popc(peers));
            __syncwarp();
        }
        __syncthreads();
        uint32_t cnt[kPer];
        uint32_t acc = 0;
#pragma unroll
        for (int j = 0; j < kPer; ++j) {
            const int d = threadIdx.x * kPer + j;
            uint32_t run = 0;
            if (d < R) {
#pragma unroll
                for (int w = 0; w < kLbWarps; ++w) {
                    const uint32_t c = s_wh[w][d];
                    s_wh[w][d] = (uint16_t)run;
                    run += c;
                }
            }
            cnt[j] = run;
            acc += run;
        }
        uint32_t dummy;
        uint32_t ex = block_exclusive_scan<kLbThreads>(acc, s_red, &dummy);
        // publish this tile's per-digit counts (inclusive right away for tile 0)
        if (tile != drop_tile) {
#pragma unroll
            for (int j = 0; j < kPer; ++j) {
                const int d = threadIdx.x * kPer + j;
                if (d < R)
                    st_release(st_cur + (size_t)tile * R + d,
                               ((tile == 0 ? kStateIncl : kStateAgg) << 32) | (uint64_t)cnt[j]);
            }
        }
        // look back for each digit: prefix_wg = sum of the lower tiles' counts
        bool ok = true;
#pragma unroll
        for (int j = 0; j < kPer; ++j) {
            const int d = threadIdx.x * kPer + j;
            uint32_t excl = 0;
            if (d < R && tile > 0) {
                for (int tp = tile - 1; tp >= 0 && ok;) {
                    uint64_t v = ld_acquire(st_cur + (size_t)tp * R + d);
                    uint32_t spins = 0;
                    while ((v >> 32) == 0) {
                        if ((spins & 63) == 0 && ld_volatile(flags + 1) != 0u) { ok = false; break; }
                        if (++spins > kMaxSpin) {
                            flags[1] = 1u;  // every writer stores the same value
                            ok = false;
                            break;
                        }
                        __nanosleep(256);
                        v = ld_acquire(st_cur + (size_t)tp * R + d);
                    }
                    if (!ok) break;
                    excl += (uint32_t)v;
                    if ((v >> 32) == kStateIncl) break;
                    --tp;
                }
            }
            if (d < R) {
                s_start[d] = ex;
                s_goff[d] = __ldg(base + d) + excl - ex;
                if (ok && tile != drop_tile && tile > 0)
                    st_release(st_cur + (size_t)tile * R + d, (kStateIncl << 32) | (uint64_t)(excl + cnt[j]));
            }
            ex += cnt[j];
        }
        if (!ok) s_ok = 0;
        __syncthreads();
        const bool tile_ok = s_ok != 0;
        if (tile_ok) {
#pragma unroll
            for (int k = 0; k < kLbItems; ++k) {
                const uint32_t d = dig[k];
                if (d < (uint32_t)R) {
                    const uint32_t p = s_start[d] + s_wh[warp][d] + rnk[k];
                    s_keys[p] = key[k];
                    s_vals[p] = val[k];
                }
            }
        }
        __syncthreads();
        if (tile_ok) {
            for (int p = threadIdx.x; p < count; p += kLbThreads) {
                const uint64_t kk = s_keys[p];
                const uint32_t d = (uint32_t)(kk >> shift) & mask;
                const uint32_t pos = s_goff[d] + p;
                if (pos < n) {
                    keys_out[pos] = kk;
                    vals_out[pos] = s_vals[p];
                }
            }
        }
        // clear this tile's words of the next pass's buffer
        for (int d = threadIdx.x; d < R; d += kLbThreads) st_next[(size_t)tile * R + d] = 0ull;
        __syncthreads();
    }
}

template <int BITS>
constexpr size_t lb_pass_smem() {
    return (size_t)kLbTile * 12 + (size_t)kLbWarps * (1 << BITS) * 2 + (size_t)(1 << BITS) * 8 +
           (kLbThreads / 32 + 1) * 4;
}

int lb_tiles(int64_t cap) { return (int)((cap + kLbTile - 1) / kLbTile); }

struct LbScratch {
    uint32_t* partials;
    uint32_t* base;
    uint64_t* st[2];
};

LbScratch lb_layout(void* scratch, int64_t cap) {
    LbScratch s;
    char* p = static_cast<char*>(scratch);
    const size_t words = (size_t)kLbMaxPasses * (1 << kLbMaxBits);
    s.partials = reinterpret_cast<uint32_t*>(p);
    p += (size_t)kLbHistBlocks * words * 4;
    s.base = reinterpret_cast<uint32_t*>(p);
    p += words * 4;
    const size_t st_words = (size_t)(lb_tiles(cap) > 0 ? lb_tiles(cap) : 1) * (1 << kLbMaxBits);
    s.st[0] = reinterpret_cast<uint64_t*>(p);
    s.st[1] = s.st[0] + st_words;
    return s;
}

template <int BITS>
cudaError_t lb_sort(const uint32_t* num_keys, int64_t cap, int begin_bit, int end_bit, uint64_t* keys,
                    uint32_t* vals, uint64_t* keys_alt, uint32_t* vals_alt, void* scratch, uint32_t* flags,
                    int drop_tile, int* in_alt, cudaStream_t stream) {
    constexpr int R = 1 << BITS;
    const int passes = (end_bit - begin_bit + BITS - 1) / BITS;
    const int tiles = lb_tiles(cap);
    LbScratch s = lb_layout(scratch, cap);
    constexpr size_t smem = lb_pass_smem<BITS>();
    int dev = 0, sms = 148, occ = 1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    static std::atomic<uint64_t> configured{0};
    const uint64_t bit = uint64_t(1) << (dev & 63);
    if (!(configured.load(std::memory_order_acquire) & bit)) {
        e = cudaFuncSetAttribute(k_lb_pass<BITS>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        configured.fetch_or(bit, std::memory_order_acq_rel);
    }
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_lb_pass<BITS>, kLbThreads, smem);
    if (e != cudaSuccess) return e;
    // Co-resident persistent grid: every block runs at once, so a tile's
    // predecessors always make progress.
    const int grid = tiles < sms * occ ? tiles : sms * occ;
    e = launch_pdl(k_lb_hist<BITS>, dim3(kLbHistBlocks), dim3(kLbThreads), (size_t)passes * R * 4, stream,
                   (const uint64_t*)keys, num_keys, begin_bit, passes, end_bit, s.partials, s.st[0],
                   (int64_t)tiles * R, flags, (uint32_t)cap);
    if (e != cudaSuccess) return e;
    e = launch_pdl(k_lb_hist_scan<BITS>, dim3(passes), dim3(R > 256 ? R : 256), 0, stream,
                   (const uint32_t*)s.partials, passes, s.base);
    if (e != cudaSuccess) return e;
    uint64_t* kin = keys;
    uint32_t* vin = vals;
    uint64_t* kout = keys_alt;
    uint32_t* vout = vals_alt;
    for (int p = 0; p < passes; ++p) {
        const int shift = begin_bit + p * BITS;
        const int bits = end_bit - shift < BITS ? end_bit - shift : BITS;
        const uint32_t mask = (1u << bits) - 1u;
        if (grid > 0) {
            e = launch_pdl(k_lb_pass<BITS>, dim3(grid), dim3(kLbThreads), smem, stream, (const uint64_t*)kin,
                           (const uint32_t*)vin, kout, vout, num_keys, shift, mask,
                           (const uint32_t*)(s.base + p * R), s.st[p & 1], s.st[(p + 1) & 1], flags,
                           p == 0 ? drop_tile : -1, (uint32_t)cap);
            if (e != cudaSuccess) return e;
        }
        uint64_t* tk = kin; kin = kout; kout = tk;
        uint32_t* tv = vin; vin = vout; vout = tv;
    }
    *in_alt = passes & 1;
    return cudaSuccess;
}

}  // namespace

bool sort_lookback_supported(int digit_bits, int begin_bit, int end_bit) {
    return digit_bits >= 4 && digit_bits <= kLbMaxBits &&
           (end_bit - begin_bit + digit_bits - 1) / digit_bits <= kLbMaxPasses;
}

size_t sort_lookback_scratch_bytes(int64_t key_capacity) {
    const size_t words = (size_t)kLbMaxPasses * (1 << kLbMaxBits);
    const size_t st_words = (size_t)(lb_tiles(key_capacity) > 0 ? lb_tiles(key_capacity) : 1) * (1 << kLbMaxBits);
    return (size_t)kLbHistBlocks * words * 4 + words * 4 + 2 * st_words * 8;
}

cudaError_t launch_sort_lookback(const uint32_t* num_keys, int64_t key_capacity, int begin_bit, int end_bit,
                                 int digit_bits, uint64_t* keys, uint32_t* vals, uint64_t* keys_alt,
                                 uint32_t* vals_alt, void* scratch, uint32_t* flags, int drop_tile, int* in_alt,
                                 cudaStream_t stream) {
    switch (digit_bits) {
        case 4: return lb_sort<4>(num_keys, key_capacity, begin_bit, end_bit, keys, vals, keys_alt, vals_alt, scratch, flags, drop_tile, in_alt, stream);
        case 5: return lb_sort<5>(num_keys, key_capacity, begin_bit, end_bit, keys, vals, keys_alt, vals_alt, scratch, flags, drop_tile, in_alt, stream);
        case 6: return lb_sort<6>(num_keys, key_capacity, begin_bit, end_bit, keys, vals, keys_alt, vals_alt, scratch, flags, drop_tile, in_alt, stream);
        case 7: return lb_sort<7>(num_keys, key_capacity, begin_bit, end_bit, keys, vals, keys_alt, vals_alt, scratch, flags, drop_tile, in_alt, stream);
        case 8: return lb_sort<8>(num_keys, key_capacity, begin_bit, end_bit, keys, vals, keys_alt, vals_alt, scratch, flags, drop_tile, in_alt, stream);
        case 9: return lb_sort<9>(num_keys, key_capacity, begin_bit, end_bit, keys, vals, keys_alt, vals_alt, scratch, flags, drop_tile, in_alt, stream);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace ws
