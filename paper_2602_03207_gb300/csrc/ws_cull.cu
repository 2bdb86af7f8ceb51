// Compaction of the surviving splats into the <tile, splat> pair list.
//
// §3.2 compacts the splats that survive culling into a buffer; this path writes one
// (tile, depth) key per overlapped tile (the tile decomposition §3.4
// describes). The slot of every pair comes from an exclusive scan of
// tiles_touched, computed wait-free in the spirit of §3.3.2's hierarchical
// scan: level 0 reduces fixed chunks, level 1 scans the chunk sums in one
// block, and level 0 again scans inside each chunk and adds its chunk
// offset. Three dispatches, no block waits for another, no global atomics.
//
// Emission is balanced over pairs rather than over Gaussians: a block owns a
// chunk of Gaussians and the contiguous slot range their pairs occupy; its
// threads walk that slot range in order, so every key/value write is
// coalesced no matter how many tiles one splat covers. A thread finds the
// Gaussian of its slot by binary search over the chunk's local offsets in
// shared memory.
#include "ws_common.cuh"
#include "ws_kernels.cuh"

namespace ws {

namespace {

constexpr int kScanThreads = 256;
constexpr int kScanItems = 4;
constexpr int kChunk = kScanThreads * kScanItems;  // Gaussians per block
constexpr int kTopThreads = 1024;
constexpr int kSlotCap = 4096;  // slots per chunk resolved through shared memory

// Pair counts are summed in 64 bits and stored saturated at 2^32 - 1: a
// frame may cover more than 2^32 pairs (screen-filling splats with the
// culling switched off), and a saturated slot is past any key capacity
// (< 2^31), so such pairs are dropped and the capacity flag is raised
// instead of wrapping around onto valid slots.
constexpr uint32_t kSlotSat = 0xffffffffu;

__device__ __forceinline__ uint32_t sat32(uint64_t v) { return v < (uint64_t)kSlotSat ? (uint32_t)v : kSlotSat; }

// Level 0 up: one sum of tiles_touched per chunk.
__global__ void __launch_bounds__(kScanThreads)
k_chunk_sums(int64_t n, const uint32_t* __restrict__ touched, uint32_t* __restrict__ sums) {
    __shared__ uint64_t s_red[kScanThreads / 32];
    pdl_wait();
    const int64_t base = (int64_t)blockIdx.x * kChunk;
    uint64_t acc = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        int64_t i = base + threadIdx.x + k * kScanThreads;
        if (i < n) acc += __ldg(touched + i);
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(kFull, acc, o);
    if (lane == 0) s_red[warp] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint64_t t = 0;
#pragma unroll
        for (int w = 0; w < kScanThreads / 32; ++w) t += s_red[w];
        sums[blockIdx.x] = sat32(t);
    }
}

// Level 1: exclusive scan of the chunk sums in one block (64-bit running
// total, chunk offsets stored saturated); total pairs, the clamped key count
// and the capacity flag.
__global__ void __launch_bounds__(kTopThreads)
k_chunk_scan(int64_t nchunks, int64_t n, uint32_t* __restrict__ sums, uint32_t* __restrict__ offsets,
             uint32_t* __restrict__ num_keys, int64_t capacity, uint32_t* __restrict__ status) {
    __shared__ uint64_t s_red[kTopThreads / 32 + 1];
    pdl_wait();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint64_t carry = 0;
    for (int64_t start = 0; start < nchunks; start += kTopThreads) {
        const int64_t c = start + threadIdx.x;
        const uint64_t v = c < nchunks ? sums[c] : 0u;
        uint64_t x = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint64_t y = __shfl_up_sync(kFull, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) s_red[warp] = x;
        __syncthreads();
        if (warp == 0) {
            const uint64_t w = s_red[lane];
            uint64_t s = w;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint64_t y = __shfl_up_sync(kFull, s, o);
                if (lane >= o) s += y;
            }
            s_red[lane] = s - w;
            if (lane == 31) s_red[32] = s;
        }
        __syncthreads();
        if (c < nchunks) sums[c] = sat32(carry + s_red[warp] + x - v);
        carry += s_red[32];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        offsets[n] = sat32(carry);
        const bool over = carry > (uint64_t)capacity;
        *num_keys = over ? (uint32_t)capacity : (uint32_t)carry;
        // This frame's status words: stored outright, so no clear is needed.
        status[0] = over ? 1u : 0u;
        status[1] = 0u;
    }
}

// Level 0 down + emission. In a batch (BATCH = true) item i is (view
// v = i / per_view, Gaussian g = i - v * per_view), its tile ids are offset
// into the global tile grid and its value is g; for one view the item is
// the Gaussian itself.
template <bool BATCH>
__global__ void __launch_bounds__(kScanThreads)
k_emit(int64_t n, const uint32_t* __restrict__ touched, const uint2* __restrict__ rect,
       const float* __restrict__ depth, const uint32_t* __restrict__ chunk_off, int tiles_x,
       uint32_t* __restrict__ offsets, uint64_t* __restrict__ keys, uint32_t* __restrict__ vals,
       int64_t capacity, uint32_t per_view, const ViewGrid grid) {
    __shared__ uint32_t s_off[kChunk + 1];
    __shared__ uint2 s_rect[kChunk];
    __shared__ uint32_t s_depth[kChunk];
    __shared__ uint32_t s_red[kScanThreads / 32 + 1];
    __shared__ __align__(16) uint16_t s_owner[kSlotCap];  // slot -> local Gaussian (fast path; < kChunk)
    pdl_wait();
    const int64_t base = (int64_t)blockIdx.x * kChunk;
    const int cnt = (int)((n - base) < kChunk ? (n - base) : kChunk);

    // Blocked arrangement: thread t owns Gaussians base + t*kScanItems .. + kScanItems - 1,
    // so a thread-serial prefix plus one block scan gives the local offsets.
    uint32_t v[kScanItems];
    uint32_t acc = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        int li = threadIdx.x * kScanItems + k;
        v[k] = li < cnt ? __ldg(touched + base + li) : 0u;
        acc += v[k];
    }
    uint32_t total;
    uint32_t ex = block_exclusive_scan<kScanThreads>(acc, s_red, &total);
    // A saturated chunk offset (2^32 - 1) puts every slot of the chunk past
    // the capacity; offsets are stored saturated likewise.
    const uint32_t coff = chunk_off[blockIdx.x];
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        int li = threadIdx.x * kScanItems + k;
        s_off[li] = ex;
        if (li < cnt) offsets[base + li] = sat32((uint64_t)coff + ex);
        ex += v[k];
    }
    if (threadIdx.x == 0) s_off[kChunk] = total;
    // Stage rect and depth of the chunk (coalesced).
    for (int li = threadIdx.x; li < cnt; li += kScanThreads) {
        s_rect[li] = __ldg(rect + base + li);
        s_depth[li] = __float_as_uint(__ldg(depth + base + li));
    }
    __syncthreads();

    // Slot -> owning Gaussian. When the chunk's slots fit in shared memory,
    // every Gaussian with tiles writes its index at its first slot and a
    // block-wide running maximum fills the rest (indices increase with
    // slots); otherwise each slot binary-searches the local offsets.
    const bool fast = total <= (uint32_t)kSlotCap;
    if (fast) {
        for (uint32_t e = threadIdx.x; e < total; e += kScanThreads) s_owner[e] = 0;
        __syncthreads();
#pragma unroll
        for (int k = 0; k < kScanItems; ++k) {
            const int li = threadIdx.x * kScanItems + k;
            // (s_off[li] < total always holds unless the chunk's counts sum
            // past 2^32 and wrap; such a frame is flagged, and the test keeps
            // the store inside the array)
            if (li < cnt && v[k] > 0 && s_off[li] < total) s_owner[s_off[li]] = (uint16_t)li;
        }
        __syncthreads();
        // running maximum over the slots: thread-serial over kSlotPer slots
        // (read and written as 16-byte vectors: a thread's slots span 32
        // bytes, so element-wise accesses of a warp would fall 8 to a bank),
        // then a block scan
        constexpr int kSlotPer = kSlotCap / kScanThreads;
        static_assert(kSlotPer == 16, "two 16-byte vectors of slots per thread");
        uint4* own4 = reinterpret_cast<uint4*>(s_owner) + threadIdx.x * 2;
        const uint4 o0 = own4[0], o1 = own4[1];
        uint32_t ow[8] = {o0.x, o0.y, o0.z, o0.w, o1.x, o1.y, o1.z, o1.w};
        uint32_t m = 0;
#pragma unroll
        for (int k = 0; k < kSlotPer; ++k) {
            const int e = threadIdx.x * kSlotPer + k;
            if (e < (int)total) m = max(m, (ow[k >> 1] >> ((k & 1) * 16)) & 0xffffu);
        }
        // exclusive block max-scan of the per-thread maxima
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
        uint32_t x = m;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(kFull, x, o);
            if (lane >= o) x = max(x, y);
        }
        __shared__ uint32_t s_wmax[kScanThreads / 32];
        if (lane == 31) s_wmax[warp] = x;
        __syncthreads();
        uint32_t before = 0;
        for (int w = 0; w < warp; ++w) before = max(before, s_wmax[w]);
        uint32_t prev = __shfl_up_sync(kFull, x, 1);
        prev = lane == 0 ? before : max(before, prev);
#pragma unroll
        for (int k = 0; k < kSlotPer; ++k) {
            const int e = threadIdx.x * kSlotPer + k;
            if (e < (int)total) {
                const int sh = (k & 1) * 16;
                prev = max(prev, (ow[k >> 1] >> sh) & 0xffffu);
                ow[k >> 1] = (ow[k >> 1] & ~(0xffffu << sh)) | (prev << sh);
            }
        }
        own4[0] = make_uint4(ow[0], ow[1], ow[2], ow[3]);
        own4[1] = make_uint4(ow[4], ow[5], ow[6], ow[7]);
        __syncthreads();
    }
    for (uint32_t s = threadIdx.x; s < total; s += kScanThreads) {
        int64_t slot = (int64_t)coff + s;
        if (slot >= capacity) break;
        int lo;
        if (fast) {
            lo = (int)s_owner[s];
        } else {
            lo = 0;
            int hi = cnt - 1;  // largest g with s_off[g] <= s
            while (lo < hi) {
                int mid = (lo + hi + 1) >> 1;
                if (s_off[mid] <= s) lo = mid; else hi = mid - 1;
            }
        }
        uint32_t j = s - s_off[lo];
        uint2 r = s_rect[lo];
        uint32_t rx0 = r.x & 0xffffu, ry0 = r.x >> 16, rx1 = r.y & 0xffffu;
        uint32_t w = rx1 - rx0 + 1;
        uint32_t dy = j / w, dx = j - dy * w;
        const uint32_t item = (uint32_t)(base + lo);
        uint64_t tile;
        uint32_t val;
        if (BATCH) {
            const uint32_t v = item / per_view;
            tile = (uint64_t)grid.tile_off[v] + (uint64_t)(ry0 + dy) * grid.tiles_x[v] + (rx0 + dx);
            val = item - v * per_view;
        } else {
            tile = (uint64_t)(ry0 + dy) * (uint64_t)tiles_x + (rx0 + dx);
            val = item;
        }
        keys[slot] = (tile << 31) | (uint64_t)(s_depth[lo] & 0x7fffffffu);
        vals[slot] = val;
    }
}

}  // namespace

size_t cull_scratch_bytes(int64_t n) {
    int64_t nchunks = (n + kChunk - 1) / kChunk;
    return (size_t)(nchunks > 0 ? nchunks : 1) * sizeof(uint32_t);
}

cudaError_t launch_cull(int64_t n, const uint32_t* tiles_touched, const uint16_t* rect,
                        const float* depth, const Frame& f, uint32_t* offsets, uint64_t* keys,
                        uint32_t* vals, int64_t key_capacity, uint32_t* num_keys,
                        uint32_t* status, void* scratch, cudaStream_t stream) {
    const int64_t nchunks = (n + kChunk - 1) / kChunk;
    uint32_t* sums = static_cast<uint32_t*>(scratch);
    cudaError_t e = cudaSuccess;
    if (nchunks > 0) {
        e = launch_pdl(k_chunk_sums, dim3((unsigned)nchunks), dim3(kScanThreads), 0, stream, n, tiles_touched, sums);
        if (e != cudaSuccess) return e;
    }
    e = launch_pdl(k_chunk_scan, dim3(1), dim3(kTopThreads), 0, stream, (int64_t)nchunks, n, sums, offsets,
                   num_keys, key_capacity, status);
    if (e != cudaSuccess) return e;
    if (nchunks > 0) {
        ViewGrid g;
        g.views = 1;
        g.tiles_x[0] = (uint32_t)f.TX;
        g.tile_off[0] = 0;
        g.tile_off[1] = (uint32_t)(f.TX * f.TY);
        e = launch_pdl(k_emit<false>, dim3((unsigned)nchunks), dim3(kScanThreads), 0, stream, n, tiles_touched,
                       reinterpret_cast<const uint2*>(rect), depth, (const uint32_t*)sums, (int)f.TX, offsets,
                       keys, vals, key_capacity, (uint32_t)(n > 0 ? n : 1), g);
    }
    return e;
}

cudaError_t launch_cull_batch(int64_t n, const ViewGrid& grid, const uint32_t* tiles_touched,
                              const uint16_t* rect, const float* depth, uint32_t* offsets, uint64_t* keys,
                              uint32_t* vals, int64_t key_capacity, uint32_t* num_keys, uint32_t* status,
                              void* scratch, cudaStream_t stream) {
    const int64_t items = n * grid.views;
    const int64_t nchunks = (items + kChunk - 1) / kChunk;
    uint32_t* sums = static_cast<uint32_t*>(scratch);
    cudaError_t e = cudaSuccess;
    if (nchunks > 0) {
        e = launch_pdl(k_chunk_sums, dim3((unsigned)nchunks), dim3(kScanThreads), 0, stream, items, tiles_touched,
                       sums);
        if (e != cudaSuccess) return e;
    }
    e = launch_pdl(k_chunk_scan, dim3(1), dim3(kTopThreads), 0, stream, (int64_t)nchunks, items, sums, offsets,
                   num_keys, key_capacity, status);
    if (e != cudaSuccess) return e;
    if (nchunks > 0) {
        e = launch_pdl(k_emit<true>, dim3((unsigned)nchunks), dim3(kScanThreads), 0, stream, items, tiles_touched,
                       reinterpret_cast<const uint2*>(rect), depth, (const uint32_t*)sums, 0, offsets, keys, vals,
                       key_capacity, (uint32_t)n, grid);
    }
    return e;
}

}  // namespace ws
