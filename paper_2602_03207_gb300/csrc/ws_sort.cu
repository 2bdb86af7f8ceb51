// Wait-free, deterministic LSD radix sort of (uint64 key, uint32 value)
// pairs (paper §3.3.2).
//
// The paper's decomposition of the scatter position of element i with
// digit d,
//     pos = base_d + rank_i,   rank_i = prefix_wg + rank_local_i,
// is kept exactly. Each pass is three dispatches:
//   1. upsweep:   every block counts the digits of its tile of keys
//                 (warp-private histograms in shared memory, warp-aggregated
//                 by a per-bit ballot match, so each distinct digit costs one
//                 update per warp instruction) and writes one column of the
//                 digit-major matrix hist[d][tile].
//   2. scan:      one block per digit scans its row; the exclusive row
//                 prefix is prefix_wg, the row total feeds base_d.
//   3. downsweep: every block re-reads its tile, ranks each key among the
//                 tile's equal digits in input order (rank_local), sorts the
//                 tile by digit in shared memory and writes each digit run
//                 to base_d + prefix_wg + position: consecutive threads write
//                 consecutive addresses.
// No block ever waits on another (no flags, no spinning) and no global
// atomics are used, so the result is identical under any scheduling; the
// order of equal keys is their input order.
//
// The key count lives in device memory (written by the compaction), so the
// grids are sized by the capacity and blocks past the count return at once.
#include <atomic>
#include <mutex>

#include "ws_common.cuh"
#include "ws_kernels.cuh"

namespace ws {

namespace {

constexpr int kSortThreads = 256;
constexpr int kSortWarps = kSortThreads / kWarp;
#ifndef WS_SORT_ITEMS
#define WS_SORT_ITEMS 8
#endif
constexpr int kSortItems = WS_SORT_ITEMS;  // keys per thread
constexpr int kSortTile = kSortThreads * kSortItems;  // keys per block


template <int BITS>
__global__ void __launch_bounds__(kSortThreads)
k_sort_upsweep(const uint64_t* __restrict__ keys, const uint32_t* __restrict__ num_keys, int shift,
               uint32_t mask, uint32_t* __restrict__ hist, int max_tiles, uint32_t cap) {
    constexpr int R = 1 << BITS;
    __shared__ uint16_t s_hist[kSortWarps][R];  // per-warp counts (<= 512 each)
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int d = threadIdx.x; d < kSortWarps * R; d += kSortThreads) (&s_hist[0][0])[d] = 0;
    pdl_wait();
    const uint32_t n = min(*num_keys, cap);
    const int tile = blockIdx.x;
    if ((int64_t)tile * kSortTile >= (int64_t)n) return;
    __syncthreads();
    const int64_t base = (int64_t)tile * kSortTile + warp * (kWarp * kSortItems);
    uint32_t dig[kSortItems];
#pragma unroll
    for (int k = 0; k < kSortItems; ++k) {
        int64_t idx = base + k * kWarp + lane;
        dig[k] = idx < n ? (uint32_t)(__ldg(keys + idx) >> shift) & mask : (uint32_t)R;
    }
#pragma unroll
    for (int k = 0; k < kSortItems; ++k) {
        const bool ok = dig[k] < (uint32_t)R;
        const uint32_t peers = warp_match_digit<BITS>(dig[k], ok);
        if (ok && lane == __ffs(peers) - 1)
            s_hist[warp][dig[k]] = (uint16_t)(s_hist[warp][dig[k]] + __popc(peers));
        __syncwarp();
    }
    __syncthreads();
    for (int d = threadIdx.x; d < R; d += kSortThreads) {
        uint32_t s = 0;
#pragma unroll
        for (int w = 0; w < kSortWarps; ++w) s += s_hist[w][d];
        hist[(size_t)d * max_tiles + tile] = s;
    }
}

// One block per digit: exclusive scan of hist[d][0 .. tiles) in place, row
// total into totals[d].
__global__ void __launch_bounds__(kSortThreads)
k_sort_scan(const uint32_t* __restrict__ num_keys, uint32_t* __restrict__ hist,
            uint32_t* __restrict__ totals, int max_tiles, uint32_t cap) {
    __shared__ uint32_t s_red[kSortThreads / 32 + 1];
    pdl_wait();
    const uint32_t n = min(*num_keys, cap);
    const int tiles = (int)((n + kSortTile - 1) / kSortTile);
    uint32_t* row = hist + (size_t)blockIdx.x * max_tiles;
    uint32_t carry = 0;
    constexpr int kPer = 4;
    for (int start = 0; start < tiles; start += kSortThreads * kPer) {
        uint32_t v[kPer];
        uint32_t acc = 0;
#pragma unroll
        for (int k = 0; k < kPer; ++k) {
            int t = start + threadIdx.x * kPer + k;
            v[k] = t < tiles ? row[t] : 0u;
            acc += v[k];
        }
        uint32_t total;
        uint32_t ex = block_exclusive_scan<kSortThreads>(acc, s_red, &total);
#pragma unroll
        for (int k = 0; k < kPer; ++k) {
            int t = start + threadIdx.x * kPer + k;
            if (t < tiles) row[t] = carry + ex;
            ex += v[k];
        }
        carry += total;
    }
    if (threadIdx.x == 0) totals[blockIdx.x] = carry;
}

template <int BITS>
__global__ void __launch_bounds__(kSortThreads)
k_sort_downsweep(const uint64_t* __restrict__ keys_in, const uint32_t* __restrict__ vals_in,
                 uint64_t* __restrict__ keys_out, uint32_t* __restrict__ vals_out,
                 const uint32_t* __restrict__ num_keys, int shift, uint32_t mask,
                 const uint32_t* __restrict__ hist, const uint32_t* __restrict__ totals,
                 int max_tiles, uint32_t cap) {
    constexpr int R = 1 << BITS;
    constexpr int kPerThread = R > kSortThreads ? R / kSortThreads : 1;
    extern __shared__ __align__(16) unsigned char s_raw[];
    uint64_t* s_keys = reinterpret_cast<uint64_t*>(s_raw);                  // [kSortTile]
    uint32_t* s_vals = reinterpret_cast<uint32_t*>(s_keys + kSortTile);     // [kSortTile]
    auto s_wh = reinterpret_cast<uint16_t (*)[R]>(s_vals + kSortTile);     // [warps][R] counts, then prefixes
    uint32_t* s_start = reinterpret_cast<uint32_t*>(&s_wh[kSortWarps][0]); // [R] tile-local run starts
    uint32_t* s_goff = s_start + R;  // [R] global position of each run minus its local start
    uint32_t* s_red = s_goff + R;    // [warps + 1]

    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int d = threadIdx.x; d < kSortWarps * R; d += kSortThreads) (&s_wh[0][0])[d] = 0;
    pdl_wait();
    const uint32_t n = min(*num_keys, cap);
    const int tile = blockIdx.x;
    const int64_t tile_base = (int64_t)tile * kSortTile;
    if (tile_base >= (int64_t)n) return;
    const int count = (int)(((int64_t)n - tile_base) < kSortTile ? ((int64_t)n - tile_base) : kSortTile);
    // Request this block's column of prefix_wg and the digit totals now, so
    // their latency overlaps the key loads and the ranking below.
    uint32_t tv[kPerThread], hv[kPerThread];
#pragma unroll
    for (int j = 0; j < kPerThread; ++j) {
        const int d = threadIdx.x * kPerThread + j;
        tv[j] = d < R ? __ldg(totals + d) : 0u;
        hv[j] = d < R ? __ldg(hist + (size_t)d * max_tiles + tile) : 0u;
    }
    __syncthreads();

    // Load in warp-striped order: item k of lane l of warp w is element
    // w*512 + k*32 + l of the tile, so (w, k, l) order is input order.
    const int64_t base = tile_base + warp * (kWarp * kSortItems);
    uint64_t key[kSortItems];
    uint32_t val[kSortItems];
    uint32_t dig[kSortItems];
    uint16_t rnk[kSortItems];
#pragma unroll
    for (int k = 0; k < kSortItems; ++k) {
        int64_t idx = base + k * kWarp + lane;
        bool ok = idx < (int64_t)n;
        key[k] = ok ? __ldg(keys_in + idx) : 0ull;
        val[k] = ok ? __ldg(vals_in + idx) : 0u;
        dig[k] = ok ? (uint32_t)(key[k] >> shift) & mask : (uint32_t)R;
    }
    // rank_local within the warp, in input order.
    const uint32_t lt = lanemask_lt();
#pragma unroll
    for (int k = 0; k < kSortItems; ++k) {
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

    // Per digit: exclusive prefix over warps, tile count, block scan over
    // digits -> tile-local run starts; global offsets base_d + prefix_wg.
    uint32_t cnt[kPerThread];
    uint32_t acc = 0;
#pragma unroll
    for (int j = 0; j < kPerThread; ++j) {
        int d = threadIdx.x * kPerThread + j;
        uint32_t run = 0;
        if (d < R) {
#pragma unroll
            for (int w = 0; w < kSortWarps; ++w) {
                uint32_t c = s_wh[w][d];
                s_wh[w][d] = (uint16_t)run;
                run += c;
            }
        }
        cnt[j] = run;
        acc += run;
    }
    uint32_t dummy;
    uint32_t ex = block_exclusive_scan<kSortThreads>(acc, s_red, &dummy);
    // base_d: exclusive scan of the digit totals of the whole pass.
    uint32_t tacc = 0;
#pragma unroll
    for (int j = 0; j < kPerThread; ++j) tacc += tv[j];
    uint32_t tex = block_exclusive_scan<kSortThreads>(tacc, s_red, &dummy);
#pragma unroll
    for (int j = 0; j < kPerThread; ++j) {
        int d = threadIdx.x * kPerThread + j;
        if (d < R) {
            s_start[d] = ex;
            s_goff[d] = tex + hv[j] - ex;
        }
        ex += cnt[j];
        tex += tv[j];
    }
    __syncthreads();

    // Sort the tile by digit in shared memory.
#pragma unroll
    for (int k = 0; k < kSortItems; ++k) {
        uint32_t d = dig[k];
        if (d < (uint32_t)R) {
            uint32_t p = s_start[d] + s_wh[warp][d] + rnk[k];
            s_keys[p] = key[k];
            s_vals[p] = val[k];
        }
    }
    __syncthreads();

    // Write each digit run to pos = base_d + prefix_wg + local position.
    for (int p = threadIdx.x; p < count; p += kSortThreads) {
        uint64_t kk = s_keys[p];
        uint32_t d = (uint32_t)(kk >> shift) & mask;
        uint32_t pos = s_goff[d] + p;
        keys_out[pos] = kk;
        vals_out[pos] = s_vals[p];
    }
}

template <int BITS>
constexpr size_t downsweep_smem() {
    return (size_t)kSortTile * 12 + (size_t)kSortWarps * (1 << BITS) * 2 + (size_t)(1 << BITS) * 8 +
           (kSortThreads / 32 + 1) * 4;
}

struct SortScratch {
    uint32_t* hist;
    uint32_t* totals;
};

int max_tiles_for(int64_t capacity) { return (int)((capacity + kSortTile - 1) / kSortTile); }

template <int BITS>
cudaError_t sort_passes(const uint32_t* num_keys, int64_t capacity, int begin_bit, int end_bit,
                        uint64_t* keys, uint32_t* vals, uint64_t* keys_alt, uint32_t* vals_alt,
                        SortScratch s, int* in_alt, cudaStream_t stream) {
    const int max_tiles = max_tiles_for(capacity);
    // A count above the capacity is clamped to it on the device (the caller
    // states it must not exceed it), so no pass writes past the key buffers,
    // the histogram rows or the totals.
    const uint32_t cap = (uint32_t)capacity;
    constexpr size_t smem = downsweep_smem<BITS>();
    // The dynamic shared-memory limit is a per-device function attribute:
    // set it once per (instantiation, device).
    static std::atomic<uint64_t> configured{0};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const uint64_t bit = uint64_t(1) << (dev & 63);
    if (!(configured.load(std::memory_order_acquire) & bit)) {
        e = cudaFuncSetAttribute(k_sort_downsweep<BITS>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        configured.fetch_or(bit, std::memory_order_acq_rel);
    }
    uint64_t* kin = keys;
    uint32_t* vin = vals;
    uint64_t* kout = keys_alt;
    uint32_t* vout = vals_alt;
    int passes = 0;
    for (int shift = begin_bit; shift < end_bit; shift += BITS) {
        const int bits = end_bit - shift < BITS ? end_bit - shift : BITS;
        const uint32_t mask = (1u << bits) - 1u;
        if (max_tiles > 0) {
            e = launch_pdl(k_sort_upsweep<BITS>, dim3(max_tiles), dim3(kSortThreads), 0, stream,
                           (const uint64_t*)kin, num_keys, shift, mask, s.hist, max_tiles, cap);
            if (e != cudaSuccess) return e;
            e = launch_pdl(k_sort_scan, dim3(1 << BITS), dim3(kSortThreads), 0, stream, num_keys, s.hist,
                           s.totals, max_tiles, cap);
            if (e != cudaSuccess) return e;
            e = launch_pdl(k_sort_downsweep<BITS>, dim3(max_tiles), dim3(kSortThreads), smem, stream,
                           (const uint64_t*)kin, (const uint32_t*)vin, kout, vout, num_keys, shift, mask,
                           (const uint32_t*)s.hist, (const uint32_t*)s.totals, max_tiles, cap);
            if (e != cudaSuccess) return e;
        }
        uint64_t* tk = kin; kin = kout; kout = tk;
        uint32_t* tv = vin; vin = vout; vout = tv;
        ++passes;
    }
    *in_alt = passes & 1;
    return cudaGetLastError();
}

}  // namespace

bool sort_digit_supported(int digit_bits) { return digit_bits >= 4 && digit_bits <= 11; }

size_t sort_scratch_bytes(int64_t key_capacity, int digit_bits) {
    const size_t R = (size_t)1 << digit_bits;
    const size_t tiles = (size_t)max_tiles_for(key_capacity);
    return (R * (tiles > 0 ? tiles : 1) + R) * sizeof(uint32_t);
}

cudaError_t launch_sort(const uint32_t* num_keys, int64_t key_capacity, int begin_bit,
                        int end_bit, int digit_bits, uint64_t* keys, uint32_t* vals,
                        uint64_t* keys_alt, uint32_t* vals_alt, void* scratch, int* in_alt,
                        cudaStream_t stream) {
    const size_t R = (size_t)1 << digit_bits;
    const size_t tiles = (size_t)max_tiles_for(key_capacity);
    SortScratch s;
    s.hist = static_cast<uint32_t*>(scratch);
    s.totals = s.hist + R * (tiles > 0 ? tiles : 1);
    switch (digit_bits) {
        case 4: return sort_passes<4>(num_keys, key_capacity, begin_bit, end_bit, keys, vals, keys_alt, vals_alt, s, in_alt, stream);
        case 5: return sort_passes<5>(num_keys, key_capacity, begin_bit, end_bit, keys, vals, keys_alt, vals_alt, s, in_alt, stream);
        case 6: return sort_passes<6>(num_keys, key_capacity, begin_bit, end_bit, keys, vals, keys_alt, vals_alt, s, in_alt, stream);
        case 7: return sort_passes<7>(num_keys, key_capacity, begin_bit, end_bit, keys, vals, keys_alt, vals_alt, s, in_alt, stream);
        case 8: return sort_passes<8>(num_keys, key_capacity, begin_bit, end_bit, keys, vals, keys_alt, vals_alt, s, in_alt, stream);
        case 9: return sort_passes<9>(num_keys, key_capacity, begin_bit, end_bit, keys, vals, keys_alt, vals_alt, s, in_alt, stream);
        case 10: return sort_passes<10>(num_keys, key_capacity, begin_bit, end_bit, keys, vals, keys_alt, vals_alt, s, in_alt, stream);
        case 11: return sort_passes<11>(num_keys, key_capacity, begin_bit, end_bit, keys, vals, keys_alt, vals_alt, s, in_alt, stream);
        default: return cudaErrorInvalidValue;
    }
}


// ---------------------------------------------------------------------------
// Allocation-free variant of launch_sort (the ws_sort_noalloc entry point).
//
// Some callers cannot allocate device memory for scratch: code that runs
// inside a host engine which owns every device allocation (a plugin handed
// only its input and output buffers), or a real-time frame loop that must
// not call cudaMalloc, which can synchronise the device and stall the frame.
// For them the sort's histogram scratch lives in the file-scope array below,
// sized for at most kNoAllocMaxKeys keys. Every GPU that loads this library
// holds the array until the process exits, and all calls on a device share
// it, so two such sorts that overlap on the GPU race on it. Nothing in it
// needs clearing between calls: each pass writes every histogram entry it
// later reads (the tiles below the key count) before reading it.
namespace {

constexpr int64_t kNoAllocMaxKeys = int64_t(1) << 23;  // 8,388,608 keys
constexpr int kNoAllocMaxTiles = (int)((kNoAllocMaxKeys + kSortTile - 1) / kSortTile);
constexpr int kNoAllocMaxDigits = 256;  // 8-bit digits at most
constexpr size_t kNoAllocWords = (size_t)kNoAllocMaxDigits * kNoAllocMaxTiles + kNoAllocMaxDigits;
// 4 MiB + 1 KiB with 2,048-key blocks (the figure the header states).
static_assert(kNoAllocWords * sizeof(uint32_t) == (size_t(4) << 20) + 1024,
              "the documented size of the allocation-free sort's scratch");

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
uint32_t* g_noalloc_ptr[kMaxDevices] = {};

}  // namespace

// 4 MiB + 1 KiB per device: the digit-major histogram matrix for
// kNoAllocMaxKeys keys plus the digit totals.
static __device__ __align__(256) uint32_t ws_sort_noalloc_scratch[kNoAllocWords];

int64_t sort_noalloc_max_keys() { return kNoAllocMaxKeys; }

size_t sort_noalloc_scratch_bytes() { return sizeof(uint32_t) * kNoAllocWords; }

cudaError_t launch_sort_noalloc(const uint32_t* num_keys, int64_t key_capacity, int begin_bit,
                                int end_bit, int digit_bits, uint64_t* keys, uint32_t* vals,
                                uint64_t* keys_alt, uint32_t* vals_alt, int* in_alt,
                                cudaStream_t stream) {
    if (key_capacity > kNoAllocMaxKeys || digit_bits > 8) return cudaErrorInvalidValue;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    uint32_t* base = nullptr;
    {
        // Set-up, once per device with that device current: the host-side
        // name of the array is not a device address, so look the address up.
        std::lock_guard<std::mutex> lock(g_noalloc_mu);
        if (!g_noalloc_ptr[dev]) {
            void* p = nullptr;
            e = cudaGetSymbolAddress(&p, ws_sort_noalloc_scratch);
            if (e != cudaSuccess) return e;
            g_noalloc_ptr[dev] = static_cast<uint32_t*>(p);
        }
        base = g_noalloc_ptr[dev];
    }
    const size_t R = (size_t)1 << digit_bits;
    const size_t tiles = (size_t)max_tiles_for(key_capacity);
    SortScratch s;
    s.hist = base;
    s.totals = base + R * (tiles > 0 ? tiles : 1);
    switch (digit_bits) {
        case 4: return sort_passes<4>(num_keys, key_capacity, begin_bit, end_bit, keys, vals, keys_alt, vals_alt, s, in_alt, stream);
        case 5: return sort_passes<5>(num_keys, key_capacity, begin_bit, end_bit, keys, vals, keys_alt, vals_alt, s, in_alt, stream);
        case 6: return sort_passes<6>(num_keys, key_capacity, begin_bit, end_bit, keys, vals, keys_alt, vals_alt, s, in_alt, stream);
        case 7: return sort_passes<7>(num_keys, key_capacity, begin_bit, end_bit, keys, vals, keys_alt, vals_alt, s, in_alt, stream);
        case 8: return sort_passes<8>(num_keys, key_capacity, begin_bit, end_bit, keys, vals, keys_alt, vals_alt, s, in_alt, stream);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace ws
