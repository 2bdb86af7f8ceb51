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

// Shared memory of a chunk's emission: the chunk's local offsets, rects and
// depths, and the slot -> Gaussian map.
struct ChunkSmem {
    uint32_t off[kChunk + 1];
    uint2 rect[kChunk];
    uint32_t depth[kChunk];
    uint32_t red[kScanThreads / 32 + 1];
    uint32_t wmax[kScanThreads / 32];
    __align__(16) uint16_t owner[kSlotCap];  // slot -> local Gaussian (fast path; < kChunk)
};

// Level 0 down for chunk blockIdx.x: the chunk's local exclusive scan of
// tiles_touched (offsets[] written, saturated), its rects and depths staged,
// and, when its slots fit in shared memory, the slot -> Gaussian map (every
// Gaussian with tiles writes its index at its first slot and a block-wide
// running maximum fills the rest: indices increase with slots). Returns the
// chunk's pair count; *coff = its first slot.
__device__ __forceinline__ uint32_t chunk_prologue(ChunkSmem& S, int64_t n, const uint32_t* __restrict__ touched,
                                                   const uint2* __restrict__ rect, const float* __restrict__ depth,
                                                   const uint32_t* __restrict__ chunk_off,
                                                   uint32_t* __restrict__ offsets, int64_t base, int cnt,
                                                   uint32_t* coff, bool* fast) {
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
    uint32_t ex = block_exclusive_scan<kScanThreads>(acc, S.red, &total);
    // A saturated chunk offset (2^32 - 1) puts every slot of the chunk past
    // the capacity; offsets are stored saturated likewise.
    *coff = chunk_off[blockIdx.x];
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        int li = threadIdx.x * kScanItems + k;
        S.off[li] = ex;
        if (li < cnt) offsets[base + li] = sat32((uint64_t)*coff + ex);
        ex += v[k];
    }
    if (threadIdx.x == 0) S.off[kChunk] = total;
    // Stage rect and depth of the chunk (coalesced).
    for (int li = threadIdx.x; li < cnt; li += kScanThreads) {
        S.rect[li] = __ldg(rect + base + li);
        S.depth[li] = __float_as_uint(__ldg(depth + base + li));
    }
    __syncthreads();

    // Slot -> owning Gaussian. When the chunk's slots fit in shared memory,
    // the running-maximum map; otherwise each slot binary-searches the local
    // offsets (slot_owner).
    *fast = total <= (uint32_t)kSlotCap;
    if (*fast) {
        for (uint32_t e = threadIdx.x; e < total; e += kScanThreads) S.owner[e] = 0;
        __syncthreads();
#pragma unroll
        for (int k = 0; k < kScanItems; ++k) {
            const int li = threadIdx.x * kScanItems + k;
            // (S.off[li] < total always holds unless the chunk's counts sum
            // past 2^32 and wrap; such a frame is flagged, and the test keeps
            // the store inside the array)
            if (li < cnt && v[k] > 0 && S.off[li] < total) S.owner[S.off[li]] = (uint16_t)li;
        }
        __syncthreads();
        // running maximum over the slots: thread-serial over kSlotPer slots
        // (read and written as 16-byte vectors: a thread's slots span 32
        // bytes, so element-wise accesses of a warp would fall 8 to a bank),
        // then a block scan
        constexpr int kSlotPer = kSlotCap / kScanThreads;
        static_assert(kSlotPer == 16, "two 16-byte vectors of slots per thread");
        uint4* own4 = reinterpret_cast<uint4*>(S.owner) + threadIdx.x * 2;
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
        if (lane == 31) S.wmax[warp] = x;
        __syncthreads();
        uint32_t before = 0;
        for (int w = 0; w < warp; ++w) before = max(before, S.wmax[w]);
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
    return total;
}

// The pair at local slot s of the chunk: its (tile << 31 | depth) key, its
// value, and its tile id. In a batch (BATCH = true) item i is (view
// v = i / per_view, Gaussian g = i - v * per_view), its tile ids are offset
// into the global tile grid and its value is g; for one view the item is
// the Gaussian itself.
template <bool BATCH>
__device__ __forceinline__ uint64_t slot_pair(const ChunkSmem& S, uint32_t s, int cnt, bool fast, int64_t base,
                                              int tiles_x, uint32_t per_view, const ViewGrid& grid, uint32_t* val,
                                              uint64_t* tile_out) {
    int lo;
    if (fast) {
        lo = (int)S.owner[s];
    } else {
        lo = 0;
        int hi = cnt - 1;  // largest g with off[g] <= s
        while (lo < hi) {
            int mid = (lo + hi + 1) >> 1;
            if (S.off[mid] <= s) lo = mid; else hi = mid - 1;
        }
    }
    const uint32_t j = s - S.off[lo];
    const uint2 r = S.rect[lo];
    const uint32_t rx0 = r.x & 0xffffu, ry0 = r.x >> 16, rx1 = r.y & 0xffffu;
    const uint32_t w = rx1 - rx0 + 1;
    const uint32_t dy = j / w, dx = j - dy * w;
    const uint32_t item = (uint32_t)(base + lo);
    uint64_t tile;
    if (BATCH) {
        const uint32_t v = item / per_view;
        tile = (uint64_t)grid.tile_off[v] + (uint64_t)(ry0 + dy) * grid.tiles_x[v] + (rx0 + dx);
        *val = item - v * per_view;
    } else {
        tile = (uint64_t)(ry0 + dy) * (uint64_t)tiles_x + (rx0 + dx);
        *val = item;
    }
    *tile_out = tile;
    return (tile << 31) | (uint64_t)(S.depth[lo] & 0x7fffffffu);
}

// Level 0 down + emission: every pair of the chunk at its slot, in slot
// order.
template <bool BATCH>
__global__ void __launch_bounds__(kScanThreads)
k_emit(int64_t n, const uint32_t* __restrict__ touched, const uint2* __restrict__ rect,
       const float* __restrict__ depth, const uint32_t* __restrict__ chunk_off, int tiles_x,
       uint32_t* __restrict__ offsets, uint64_t* __restrict__ keys, uint32_t* __restrict__ vals,
       int64_t capacity, uint32_t per_view, const ViewGrid grid) {
    __shared__ ChunkSmem S;
    pdl_wait();
    const int64_t base = (int64_t)blockIdx.x * kChunk;
    const int cnt = (int)((n - base) < kChunk ? (n - base) : kChunk);
    uint32_t coff;
    bool fast;
    const uint32_t total = chunk_prologue(S, n, touched, rect, depth, chunk_off, offsets, base, cnt, &coff, &fast);
    for (uint32_t s = threadIdx.x; s < total; s += kScanThreads) {
        const int64_t slot = (int64_t)coff + s;
        if (slot >= capacity) break;
        uint32_t val;
        uint64_t tile;
        const uint64_t key = slot_pair<BATCH>(S, s, cnt, fast, base, tiles_x, per_view, grid, &val, &tile);
        keys[slot] = key;
        vals[slot] = val;
    }
}

// ---------------------------------------------------------------------------
// Compaction fused with the first partition pass of the segmented tile sort
// (one view).
//
// That sort first partitions the pairs stably by the low D bits of the tile
// id (key bits [31, 31 + D)). Here the compaction writes every pair straight
// to its place in that partition: a count of each chunk's pairs per digit
// (k_chunk_hist, from the rectangles: one row of a rectangle covers a cyclic
// run of digits), an exclusive scan of each digit's counts over the chunks
// (k_digit_scan), and an emission that ranks each pair among the chunk's
// pairs of its digit in slot order and scatters it to
//     base_d + (pairs of digit d in earlier chunks) + rank,
// with base_d the pairs of smaller digits. That is the stable partition of
// the slot-ordered list, bit for bit what the sort's first pass makes of it.
// No block waits for another and no global atomics are used. When the frame
// has more pairs than the key capacity the emission falls back to slot order
// (the first `capacity` slots, as k_emit) and the frame is flagged.

constexpr int kPartMaxBits = 8;                        // widest first-pass digit fused here
constexpr int kPartMaxDigits = 1 << kPartMaxBits;
constexpr int kPartItems = 4;                          // pairs per thread and round
constexpr int kPartRound = kScanThreads * kPartItems;  // pairs per round

// Per chunk: the pair count (as k_chunk_sums) and hist[d * nchunks + chunk],
// the chunk's pairs per digit d = tile id & (2^B - 1). A rectangle row
// y, x0..x1 covers tile ids y * tiles_x + x0 .. + x1: (x1 - x0 + 1) >> B
// full turns of the digits and a cyclic run of the remainder, added to a
// difference array in shared memory (integer additions: the counts do not
// depend on their order).
template <int B>
__global__ void __launch_bounds__(kScanThreads)
k_chunk_hist(int64_t n, const uint32_t* __restrict__ touched, const uint2* __restrict__ rect, int tiles_x,
             uint32_t* __restrict__ sums, uint32_t* __restrict__ hist, int64_t nchunks) {
    constexpr int R = 1 << B;
    __shared__ int s_diff[R + 1];
    __shared__ uint32_t s_full;
    __shared__ uint64_t s_red[kScanThreads / 32];
    __shared__ uint32_t s_scan[kScanThreads / 32 + 1];
    for (int d = threadIdx.x; d <= R; d += kScanThreads) s_diff[d] = 0;
    if (threadIdx.x == 0) s_full = 0u;
    pdl_wait();
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * kChunk;
    uint64_t acc = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        const int64_t i = base + threadIdx.x + k * kScanThreads;
        if (i >= n) continue;
        const uint32_t t = __ldg(touched + i);
        acc += t;
        if (t == 0u) continue;
        const uint2 r = __ldg(rect + i);
        const uint32_t x0 = r.x & 0xffffu, y0 = r.x >> 16, x1 = r.y & 0xffffu, y1 = r.y >> 16;
        const uint32_t w = x1 - x0 + 1, full = w >> B, rem = w & (R - 1);
        if (full) atomicAdd(&s_full, full * (y1 - y0 + 1));
        if (rem) {
            for (uint32_t y = y0; y <= y1; ++y) {
                const uint32_t st = (y * (uint32_t)tiles_x + x0) & (R - 1);
                const uint32_t en = st + rem;
                atomicAdd(&s_diff[st], 1);
                if (en <= (uint32_t)R) {
                    atomicAdd(&s_diff[en], -1);
                } else {  // the run wraps past the last digit
                    atomicAdd(&s_diff[0], 1);
                    atomicAdd(&s_diff[en - R], -1);
                }
            }
        }
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
    // counts = inclusive prefix of the difference array, plus the full turns
    constexpr int kPer = R > kScanThreads ? R / kScanThreads : 1;
    int dv[kPer];
    int a = 0;
#pragma unroll
    for (int j = 0; j < kPer; ++j) {
        const int d = threadIdx.x * kPer + j;
        dv[j] = d < R ? s_diff[d] : 0;
        a += dv[j];
    }
    uint32_t all;
    int run = (int)block_exclusive_scan<kScanThreads>((uint32_t)a, s_scan, &all);
    const uint32_t full = s_full;
#pragma unroll
    for (int j = 0; j < kPer; ++j) {
        const int d = threadIdx.x * kPer + j;
        run += dv[j];
        if (d < R) hist[(size_t)d * nchunks + blockIdx.x] = (uint32_t)run + full;
    }
}

// One block per digit: exclusive scan of hist[d][0 .. nchunks) in place,
// the row total into totals[d].
__global__ void __launch_bounds__(kScanThreads)
k_digit_scan(uint32_t* __restrict__ hist, uint32_t* __restrict__ totals, int64_t nchunks) {
    __shared__ uint32_t s_red[kScanThreads / 32 + 1];
    pdl_wait();
    uint32_t* row = hist + (size_t)blockIdx.x * nchunks;
    uint32_t carry = 0;
    constexpr int kPer = 4;
    for (int64_t start = 0; start < nchunks; start += kScanThreads * kPer) {
        uint32_t v[kPer];
        uint32_t acc = 0;
#pragma unroll
        for (int k = 0; k < kPer; ++k) {
            const int64_t t = start + threadIdx.x * kPer + k;
            v[k] = t < nchunks ? row[t] : 0u;
            acc += v[k];
        }
        uint32_t total;
        uint32_t ex = block_exclusive_scan<kScanThreads>(acc, s_red, &total);
#pragma unroll
        for (int k = 0; k < kPer; ++k) {
            const int64_t t = start + threadIdx.x * kPer + k;
            if (t < nchunks) row[t] = carry + ex;
            ex += v[k];
        }
        carry += total;
    }
    if (threadIdx.x == 0) totals[blockIdx.x] = carry;
}

// Level 0 down + emission into the first partition of the tile sort (see
// above): rounds of kPartRound slots, item k of lane l of warp w holding
// slot w * 128 + k * 32 + l of the round, so (w, k, l) order is slot order.
// Each round is ranked, sorted by digit in shared memory and written out as
// one run per digit (consecutive threads, consecutive addresses).
template <int B>
__global__ void __launch_bounds__(kScanThreads)
k_emit_part(int64_t n, const uint32_t* __restrict__ touched, const uint2* __restrict__ rect,
            const float* __restrict__ depth, const uint32_t* __restrict__ chunk_off, int tiles_x,
            uint32_t* __restrict__ offsets, uint64_t* __restrict__ keys, uint32_t* __restrict__ vals,
            int64_t capacity, const uint32_t* __restrict__ hist, const uint32_t* __restrict__ totals,
            int64_t nchunks, const uint32_t* __restrict__ status) {
    constexpr int R = 1 << B;
    constexpr int W = kScanThreads / 32;
    constexpr int kPer = R > kScanThreads ? R / kScanThreads : 1;
    __shared__ ChunkSmem S;
    __shared__ uint64_t s_k[kPartRound];  // the round's pairs, sorted by digit
    __shared__ uint32_t s_v[kPartRound];
    __shared__ uint16_t s_wc[W][R];       // per-warp digit counts, then prefixes over warps
    __shared__ uint32_t s_base[R];        // next output position of digit d for this chunk
    __shared__ uint32_t s_round[R];       // the round's count of digit d
    __shared__ uint32_t s_lstart[R];      // the round's run of digit d starts here in s_k
    __shared__ uint32_t s_red2[W + 1];
    pdl_wait();
    const int64_t base = (int64_t)blockIdx.x * kChunk;
    const int cnt = (int)((n - base) < kChunk ? (n - base) : kChunk);
    const bool over = status[0] != 0u;  // more pairs than the capacity: slot order
    // base_d (an exclusive scan of the digit totals) + this chunk's prefix
    {
        uint32_t tv[kPer], tacc = 0;
#pragma unroll
        for (int j = 0; j < kPer; ++j) {
            const int d = threadIdx.x * kPer + j;
            tv[j] = d < R ? __ldg(totals + d) : 0u;
            tacc += tv[j];
        }
        uint32_t all;
        uint32_t tex = block_exclusive_scan<kScanThreads>(tacc, s_red2, &all);
#pragma unroll
        for (int j = 0; j < kPer; ++j) {
            const int d = threadIdx.x * kPer + j;
            if (d < R) s_base[d] = tex + __ldg(hist + (size_t)d * nchunks + blockIdx.x);
            tex += tv[j];
        }
    }
    uint32_t coff;
    bool fast;
    const uint32_t total = chunk_prologue(S, n, touched, rect, depth, chunk_off, offsets, base, cnt, &coff, &fast);
    if (over) {
        for (uint32_t s = threadIdx.x; s < total; s += kScanThreads) {
            const int64_t slot = (int64_t)coff + s;
            if (slot >= capacity) break;
            uint32_t val;
            uint64_t tile;
            const uint64_t key = slot_pair<false>(S, s, cnt, fast, base, tiles_x, 1u, ViewGrid{}, &val, &tile);
            keys[slot] = key;
            vals[slot] = val;
        }
        return;
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t lt = lanemask_lt();
    for (uint32_t r0 = 0; r0 < total; r0 += kPartRound) {
        const int rcount = (int)min((uint32_t)kPartRound, total - r0);
        for (int i = threadIdx.x; i < W * R; i += kScanThreads) (&s_wc[0][0])[i] = 0;
        __syncthreads();
        uint64_t key[kPartItems];
        uint32_t val[kPartItems], dig[kPartItems], rnk[kPartItems];
#pragma unroll
        for (int k = 0; k < kPartItems; ++k) {
            const uint32_t s = r0 + warp * (32 * kPartItems) + k * 32 + lane;
            const bool ok = s < total;
            uint64_t tile = 0;
            key[k] = 0;
            val[k] = 0;
            if (ok) key[k] = slot_pair<false>(S, s, cnt, fast, base, tiles_x, 1u, ViewGrid{}, &val[k], &tile);
            dig[k] = ok ? (uint32_t)tile & (R - 1) : (uint32_t)R;
        }
        // rank among the warp's earlier pairs of the same digit
#pragma unroll
        for (int k = 0; k < kPartItems; ++k) {
            const bool ok = dig[k] < (uint32_t)R;
            const uint32_t peers = warp_match_digit<B>(ok ? dig[k] : 0u, ok);
            const int leader = __ffs(peers) - 1;
            uint32_t prior = 0;
            if (ok && lane == leader) prior = s_wc[warp][dig[k]];
            prior = __shfl_sync(kFull, prior, leader);
            rnk[k] = prior + __popc(peers & lt);
            if (ok && lane == leader) s_wc[warp][dig[k]] = (uint16_t)(prior + __popc(peers));
            __syncwarp();
        }
        __syncthreads();
        // per digit: exclusive prefix over the warps, the round's count, and
        // the start of its run in the round (a block scan over the digits)
        uint32_t rc[kPer], acc = 0;
#pragma unroll
        for (int j = 0; j < kPer; ++j) {
            const int d = threadIdx.x * kPer + j;
            uint32_t run = 0;
            if (d < R) {
#pragma unroll
                for (int w = 0; w < W; ++w) {
                    const uint32_t c = s_wc[w][d];
                    s_wc[w][d] = (uint16_t)run;
                    run += c;
                }
            }
            rc[j] = run;
            acc += run;
        }
        uint32_t all;
        uint32_t ex = block_exclusive_scan<kScanThreads>(acc, s_red2, &all);
#pragma unroll
        for (int j = 0; j < kPer; ++j) {
            const int d = threadIdx.x * kPer + j;
            if (d < R) {
                s_lstart[d] = ex;
                s_round[d] = rc[j];
            }
            ex += rc[j];
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < kPartItems; ++k) {
            if (dig[k] < (uint32_t)R) {
                const uint32_t p = s_lstart[dig[k]] + s_wc[warp][dig[k]] + rnk[k];
                s_k[p] = key[k];
                s_v[p] = val[k];
            }
        }
        __syncthreads();
        // out, one run per digit
        for (int p = threadIdx.x; p < rcount; p += kScanThreads) {
            const uint64_t kk = s_k[p];
            const uint32_t d = (uint32_t)(kk >> 31) & (R - 1);
            const uint32_t pos = s_base[d] + ((uint32_t)p - s_lstart[d]);
            if ((int64_t)pos < capacity) {
                keys[pos] = kk;
                vals[pos] = s_v[p];
            }
        }
        __syncthreads();
#pragma unroll
        for (int j = 0; j < kPer; ++j) {
            const int d = threadIdx.x * kPer + j;
            if (d < R) s_base[d] += s_round[d];
        }
        // (the next round's first barrier orders these updates before use)
    }
}

}  // namespace

size_t cull_partition_scratch_bytes(int64_t n) {
    const int64_t nchunks = (n + kChunk - 1) / kChunk;
    return ((size_t)(nchunks > 0 ? nchunks : 1) + 1) * kPartMaxDigits * sizeof(uint32_t);
}

bool cull_partition_supported(int digit_bits) { return digit_bits >= 4 && digit_bits <= kPartMaxBits; }

cudaError_t launch_cull_partition(int64_t n, const uint32_t* tiles_touched, const uint16_t* rect, const float* depth,
                                  const Frame& f, int digit_bits, uint32_t* offsets, uint64_t* keys, uint32_t* vals,
                                  int64_t key_capacity, uint32_t* num_keys, uint32_t* status, void* scratch,
                                  void* part_scratch, cudaStream_t stream) {
    const int64_t nchunks = (n + kChunk - 1) / kChunk;
    uint32_t* sums = static_cast<uint32_t*>(scratch);
    uint32_t* hist = static_cast<uint32_t*>(part_scratch);
    uint32_t* totals = hist + (size_t)(nchunks > 0 ? nchunks : 1) * kPartMaxDigits;
    const uint2* r2 = reinterpret_cast<const uint2*>(rect);
    cudaError_t e = cudaSuccess;
    auto run = [&](auto hist_kernel, auto emit_kernel, int R) -> cudaError_t {
        cudaError_t err = cudaSuccess;
        if (nchunks > 0) {
            err = launch_pdl(hist_kernel, dim3((unsigned)nchunks), dim3(kScanThreads), 0, stream, n, tiles_touched,
                             r2, (int)f.TX, sums, hist, nchunks);
            if (err != cudaSuccess) return err;
        }
        err = launch_pdl(k_chunk_scan, dim3(1), dim3(kTopThreads), 0, stream, (int64_t)nchunks, n, sums, offsets,
                         num_keys, key_capacity, status);
        if (err != cudaSuccess || nchunks == 0) return err;
        err = launch_pdl(k_digit_scan, dim3(R), dim3(kScanThreads), 0, stream, hist, totals, nchunks);
        if (err != cudaSuccess) return err;
        return launch_pdl(emit_kernel, dim3((unsigned)nchunks), dim3(kScanThreads), 0, stream, n, tiles_touched, r2,
                          depth, (const uint32_t*)sums, (int)f.TX, offsets, keys, vals, key_capacity,
                          (const uint32_t*)hist, (const uint32_t*)totals, nchunks, (const uint32_t*)status);
    };
    switch (digit_bits) {
        case 4: e = run(k_chunk_hist<4>, k_emit_part<4>, 16); break;
        case 5: e = run(k_chunk_hist<5>, k_emit_part<5>, 32); break;
        case 6: e = run(k_chunk_hist<6>, k_emit_part<6>, 64); break;
        case 7: e = run(k_chunk_hist<7>, k_emit_part<7>, 128); break;
        case 8: e = run(k_chunk_hist<8>, k_emit_part<8>, 256); break;
        default: return cudaErrorInvalidValue;
    }
    return e;
}

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
