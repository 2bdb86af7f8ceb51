// Segmented variant of the wait-free radix sort for keys whose high bits are
// a small segment id (the tile) and whose low 31 bits are a sub-key (the
// view depth), as the renderer packs them (§3.3).
//
// The result is the same stable sort of the whole key as the plain LSD sort:
//   1. partition: the wait-free LSD passes of ws_sort.cu over the segment
//      bits [31, end_bit) only. Being stable, they leave each segment's keys
//      in input order.
//   2. bounds:    start[s] = first position whose segment id is >= s, for
//      every s in [0, 2^(end_bit - 31)], from adjacent-key comparisons.
//   3. local:     every segment is sorted by its sub-key bits [begin_bit, 31)
//      on chip. A warp sorts a segment of at most 256 keys with a bitonic
//      network in registers over (sub-key << 32 | input index), whose
//      values are unique, so ties keep their input order. A block of its
//      own sorts a segment of at most 2048 keys in shared memory, and one
//      of more keys with chunked passes over global memory; both use stable
//      8-bit counting passes ranked with warp ballots, skipping a pass whose
//      digit is the same for every key of the segment.
// A stable partition by the high bits followed by a stable sort of each
// segment by the low bits orders the pairs exactly as the full-key LSD
// sort does, ties included. There are no global atomics and no block waits
// on another: each segment belongs to one block.
#include "ws_common.cuh"
#include "ws_kernels.cuh"

namespace ws {

namespace {

constexpr int kSegThreads = 256;
constexpr int kSegWarps = kSegThreads / kWarp;
constexpr int kSegItems = 8;
constexpr int kWarpCap = kWarp * kSegItems;       // keys a warp sorts alone
constexpr int kCtaCap = kSegThreads * kSegItems;  // keys the block sorts in shared memory
constexpr int kLocalBits = 8;
constexpr int kLocalRadix = 1 << kLocalBits;
constexpr int kSplitBit = 31;                     // segment id above, sub-key below
constexpr int kMaxSegBits = 24;

// start[s] for s in (seg(i-1), seg(i)]: the first position of every segment,
// empty ones included; start[nseg] = n (scan_boundaries over positions 0..n).
__global__ void __launch_bounds__(256)
k_seg_bounds(const uint64_t* __restrict__ keys, const uint32_t* __restrict__ num_keys, uint32_t cap,
             uint32_t seg_mask, uint32_t nseg, uint32_t* __restrict__ start, uint2* __restrict__ ranges,
             uint32_t ntiles) {
    pdl_wait();
    const int lane = threadIdx.x & 31;
    const int64_t nt = ranges ? (int64_t)ntiles : 0;
    scan_boundaries<4>(
        keys, min(*num_keys, cap), (int64_t)nseg,
        [seg_mask](uint64_t k) { return (int64_t)((uint32_t)(k >> kSplitBit) & seg_mask); },
        [&](int64_t lo, int64_t hi, uint32_t pos) {
            for (int64_t s = lo + 1 + lane; s <= hi; s += kWarp) start[s] = pos;
            // the same boundaries as [start, end) per segment: a local sort
            // keeps every segment in place
            for (int64_t t = lo + lane; t <= hi && t < nt; t += kWarp) {
                if (t >= 0 && t < hi) ranges[t].y = pos;
                if (t > lo) ranges[t].x = pos;
            }
        });
}

__device__ __forceinline__ uint32_t sub_key(uint64_t k, int begin_bit, uint32_t sub_mask) {
    return (uint32_t)(k >> begin_bit) & sub_mask;
}

__device__ __forceinline__ uint32_t warp_and(uint32_t v) {
    for (int o = 16; o > 0; o >>= 1) v &= __shfl_xor_sync(kFull, v, o);
    return v;
}

__device__ __forceinline__ uint32_t warp_or(uint32_t v) {
    for (int o = 16; o > 0; o >>= 1) v |= __shfl_xor_sync(kFull, v, o);
    return v;
}

// Rank items k < kn of this warp (input order k*32 + lane) among equal
// digits: rnk = earlier equal digits of the warp; cnt[d] += the warp's count.
__device__ __forceinline__ void warp_rank(const uint64_t (&key)[kSegItems], int kn, int valid_base, int n,
                                          int shift, uint32_t mask, uint32_t* cnt, uint32_t (&rnk)[kSegItems]) {
    const int lane = threadIdx.x & 31;
    const uint32_t lt = lanemask_lt();
#pragma unroll
    for (int k = 0; k < kSegItems; ++k) {
        if (k >= kn) break;
        const bool ok = valid_base + k * kWarp + lane < n;
        const uint32_t d = ok ? (uint32_t)(key[k] >> shift) & mask : 0u;
        const uint32_t peers = warp_match_digit<kLocalBits>(d, ok);
        // every lane of a digit group reads the group's running count (one
        // broadcast address per group); its first lane then advances it
        const uint32_t prior = ok ? cnt[d] : 0u;
        rnk[k] = prior + __popc(peers & lt);
        __syncwarp();  // every read before the update
        if (ok && (peers & lt) == 0u) cnt[d] = prior + __popc(peers);
        __syncwarp();
    }
}

__device__ __forceinline__ uint64_t shfl_xor64(uint64_t v, int m) {
    const uint32_t lo = __shfl_xor_sync(kFull, (uint32_t)v, m);
    const uint32_t hi = __shfl_xor_sync(kFull, (uint32_t)(v >> 32), m);
    return ((uint64_t)hi << 32) | lo;
}

// Bitonic sorting network over the warp's 32*K values, element e = lane*K + k
// in register k of lane `lane`; ascending on return. The values are
// distinct (the sort key carries the input index), so each compare-exchange
// is one 64-bit comparison whose outcome, xor the direction, picks the
// element to keep. For the stages whose partner is in another lane
// (j >= K), the direction depends on the lane only: bits j and `size` of
// e = lane*K + k are those of lane*K, since k < K <= j.
template <int K>
__device__ __forceinline__ void warp_bitonic(uint64_t (&v)[K]) {
    const int lane = threadIdx.x & 31;
    const int lk = lane * K;
    constexpr int N = kWarp * K;
#pragma unroll
    for (int size = 2; size <= N; size <<= 1) {
#pragma unroll
        for (int j = size >> 1; j > 0; j >>= 1) {
            if (j < K) {  // partner in the same lane
#pragma unroll
                for (int k = 0; k < K; ++k) {
                    if (k & j) continue;
                    const bool up = ((lk + k) & size) == 0;
                    const uint64_t x = v[k], y = v[k | j];
                    const bool swap = (x > y) == up;
                    v[k] = swap ? y : x;
                    v[k | j] = swap ? x : y;
                }
            } else {  // partner in lane ^ (j / K), same register
                const bool keep_min = ((lk & j) == 0) == ((lk & size) == 0);
#pragma unroll
                for (int k = 0; k < K; ++k) {
                    const uint64_t o = shfl_xor64(v[k], j / K);
                    v[k] = ((o < v[k]) == keep_min) ? o : v[k];
                }
            }
        }
    }
}

// Index of element e in a warp's staging slice: one padding element after
// every 8, so the transposing accesses (lane l touching element l*K + k)
// fall in distinct banks: word 9l + k for K = 8.
__device__ __forceinline__ int spad(int e) { return e + (e >> 3); }

// One warp sorts n <= 32*K pairs [b, b + n) of (kin, vin) into (kout, vout):
// the pairs are staged in the warp's slice of shared memory (keys and sort
// indices padded, see spad), the network sorts (sub-key << 32 | input index)
// -- unique values, so equal sub-keys keep their input order -- and the pairs
// are written out in that order.
template <int K>
__device__ void warp_sort(const uint64_t* kin, const uint32_t* vin, uint64_t* kout, uint32_t* vout, uint32_t b,
                          int n, int begin_bit, uint64_t* buf_k, uint32_t* buf_v, uint32_t* buf_i) {
    const int lane = threadIdx.x & 31;
    const uint32_t sub_mask = (1u << (kSplitBit - begin_bit)) - 1u;
#pragma unroll
    for (int k = 0; k < K; ++k) {
        const int idx = k * kWarp + lane;
        if (idx < n) {
            buf_k[spad(idx)] = __ldg(kin + b + idx);
            buf_v[idx] = __ldg(vin + b + idx);
        }
    }
    __syncwarp();
    uint64_t v[K];
#pragma unroll
    for (int k = 0; k < K; ++k) {
        const int e = lane * K + k;
        v[k] = e < n ? ((uint64_t)sub_key(buf_k[spad(e)], begin_bit, sub_mask) << 32) | (uint32_t)e : ~0ull;
    }
    warp_bitonic<K>(v);
#pragma unroll
    for (int k = 0; k < K; ++k) {
        const int e = lane * K + k;
        if (e < n) buf_i[spad(e)] = (uint32_t)v[k];
    }
    __syncwarp();
#pragma unroll
    for (int k = 0; k < K; ++k) {
        const int p = k * kWarp + lane;
        if (p < n) {
            const uint32_t src = buf_i[spad(p)];
            kout[b + p] = buf_k[spad((int)src)];
            vout[b + p] = buf_v[src];
        }
    }
}

// Block-wide AND / OR of one value per thread.
__device__ __forceinline__ uint32_t block_varying(uint32_t a, uint32_t o, uint32_t* red) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    a = warp_and(a);
    o = warp_or(o);
    __syncthreads();
    if (lane == 0) {
        red[2 * warp] = a;
        red[2 * warp + 1] = o;
    }
    __syncthreads();
    uint32_t ra = ~0u, ro = 0u;
#pragma unroll
    for (int w = 0; w < kSegWarps; ++w) {
        ra &= red[2 * w];
        ro |= red[2 * w + 1];
    }
    return ra ^ ro;
}

// After warp_rank by every warp: turns cnt[w][d] (warp counts) into the
// warp's first position for digit d within this chunk (digit start + the
// counts of earlier warps) and returns the chunk's count of digit
// d = threadIdx.x in *total. Threads are digits (256 threads, 256 digits).
__device__ __forceinline__ uint32_t chunk_offsets(uint32_t (*cnt)[kLocalRadix], uint32_t* red, uint32_t* total) {
    const int d = threadIdx.x;
    uint32_t run = 0;
#pragma unroll
    for (int w = 0; w < kSegWarps; ++w) {
        const uint32_t c = cnt[w][d];
        cnt[w][d] = run;
        run += c;
    }
    uint32_t all;
    const uint32_t start = block_exclusive_scan<kSegThreads>(run, red, &all);
#pragma unroll
    for (int w = 0; w < kSegWarps; ++w) cnt[w][d] += start;
    *total = run;
    return start;
}

// The block sorts 256 < n <= 2048 pairs in shared memory with 8-bit LSD
// passes; with kn = ceil(n / 256), element w*32*kn + k*32 + lane lives in
// lane `lane` of warp w, item k.
__device__ void block_sort_smem(const uint64_t* kin, const uint32_t* vin, uint64_t* kout, uint32_t* vout,
                                uint32_t b, int n, int begin_bit, uint64_t* s_key, uint32_t* s_val,
                                uint32_t (*cnt)[kLocalRadix], uint32_t* red) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    // every warp takes kn consecutive runs of 32 (input order = warp, item, lane)
    const int kn = (n + kSegThreads - 1) / kSegThreads;
    const int wbase = warp * kWarp * kn;
    const uint32_t sub_mask = (1u << (kSplitBit - begin_bit)) - 1u;
    uint64_t key[kSegItems];
    uint32_t val[kSegItems];
    uint32_t all_and = ~0u, all_or = 0u;
#pragma unroll
    for (int k = 0; k < kSegItems; ++k) {
        key[k] = 0;
        val[k] = 0;
        const int idx = wbase + k * kWarp + lane;
        if (k < kn && idx < n) {
            key[k] = __ldg(kin + b + idx);
            val[k] = __ldg(vin + b + idx);
            const uint32_t s = sub_key(key[k], begin_bit, sub_mask);
            all_and &= s;
            all_or |= s;
        }
    }
    const uint32_t varying = block_varying(all_and, all_or, red);
    for (int shift = begin_bit; shift < kSplitBit; shift += kLocalBits) {
        const int bits = kSplitBit - shift < kLocalBits ? kSplitBit - shift : kLocalBits;
        const uint32_t mask = (1u << bits) - 1u;
        if (((varying >> (shift - begin_bit)) & mask) == 0u) continue;
        for (int i = threadIdx.x; i < kSegWarps * kLocalRadix; i += kSegThreads) (&cnt[0][0])[i] = 0u;
        __syncthreads();
        uint32_t rnk[kSegItems];
        warp_rank(key, kn, wbase, n, shift, mask, cnt[warp], rnk);
        __syncthreads();
        uint32_t total;
        chunk_offsets(cnt, red, &total);
        __syncthreads();
#pragma unroll
        for (int k = 0; k < kSegItems; ++k) {
            if (k >= kn) break;
            if (wbase + k * kWarp + lane < n) {
                const uint32_t pos = cnt[warp][(uint32_t)(key[k] >> shift) & mask] + rnk[k];
                s_key[pos] = key[k];
                s_val[pos] = val[k];
            }
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < kSegItems; ++k) {
            if (k >= kn) break;
            const int idx = wbase + k * kWarp + lane;
            if (idx < n) {
                key[k] = s_key[idx];
                val[k] = s_val[idx];
            }
        }
        __syncthreads();
    }
#pragma unroll
    for (int k = 0; k < kSegItems; ++k) {
        if (k >= kn) break;
        const int idx = wbase + k * kWarp + lane;
        if (idx < n) {
            kout[b + idx] = key[k];
            vout[b + idx] = val[k];
        }
    }
}

// The block sorts n > 2048 pairs through global memory, 2048 at a time:
// per pass a histogram sweep, then chunks in order, each scattered to its
// digit's running offset. Ping-pongs between the two buffers' [b, b + n);
// the result ends in (kout, vout). Loads here are plain (not read-only
// cache): the block reads what it wrote, ordered by __syncthreads.
__device__ void block_sort_global(uint64_t* kin, uint32_t* vin, uint64_t* kout, uint32_t* vout, uint32_t b,
                                  uint32_t n, int begin_bit, uint32_t (*cnt)[kLocalRadix], uint32_t* off,
                                  uint32_t* red) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int wbase = warp * kWarpCap;
    const uint32_t sub_mask = (1u << (kSplitBit - begin_bit)) - 1u;
    uint32_t all_and = ~0u, all_or = 0u;
    for (uint32_t c0 = 0; c0 < n; c0 += kCtaCap) {
#pragma unroll
        for (int k = 0; k < kSegItems; ++k) {
            const uint32_t idx = c0 + wbase + k * kWarp + lane;
            if (idx < n) {
                const uint32_t s = sub_key(kin[b + idx], begin_bit, sub_mask);
                all_and &= s;
                all_or |= s;
            }
        }
    }
    const uint32_t varying = block_varying(all_and, all_or, red);
    uint64_t* sk = kin + b;
    uint32_t* sv = vin + b;
    uint64_t* dk = kout + b;
    uint32_t* dv = vout + b;
    bool in_out = false;  // data currently in (kout, vout)?
    for (int shift = begin_bit; shift < kSplitBit; shift += kLocalBits) {
        const int bits = kSplitBit - shift < kLocalBits ? kSplitBit - shift : kLocalBits;
        const uint32_t mask = (1u << bits) - 1u;
        if (((varying >> (shift - begin_bit)) & mask) == 0u) continue;
        // digit totals of the segment -> running offsets
        for (int i = threadIdx.x; i < kSegWarps * kLocalRadix; i += kSegThreads) (&cnt[0][0])[i] = 0u;
        __syncthreads();
        for (uint32_t c0 = 0; c0 < n; c0 += kCtaCap) {
            const int rem = (int)(n - c0 < (uint32_t)kCtaCap ? n - c0 : (uint32_t)kCtaCap);
            uint64_t key[kSegItems];
            const int kn = rem > wbase ? ((rem - wbase + kWarp - 1) / kWarp < kSegItems
                                              ? (rem - wbase + kWarp - 1) / kWarp
                                              : kSegItems)
                                       : 0;
#pragma unroll
            for (int k = 0; k < kSegItems; ++k) {
                const int idx = wbase + k * kWarp + lane;
                key[k] = (k < kn && idx < rem) ? sk[c0 + idx] : 0ull;
            }
            uint32_t rnk[kSegItems];
            warp_rank(key, kn, wbase, rem, shift, mask, cnt[warp], rnk);
        }
        __syncthreads();
        {
            const int d = threadIdx.x;
            uint32_t t = 0;
#pragma unroll
            for (int w = 0; w < kSegWarps; ++w) t += cnt[w][d];
            uint32_t all;
            off[d] = block_exclusive_scan<kSegThreads>(t, red, &all);
        }
        __syncthreads();
        for (uint32_t c0 = 0; c0 < n; c0 += kCtaCap) {
            const int rem = (int)(n - c0 < (uint32_t)kCtaCap ? n - c0 : (uint32_t)kCtaCap);
            const int kn = rem > wbase ? ((rem - wbase + kWarp - 1) / kWarp < kSegItems
                                              ? (rem - wbase + kWarp - 1) / kWarp
                                              : kSegItems)
                                       : 0;
            for (int i = threadIdx.x; i < kSegWarps * kLocalRadix; i += kSegThreads) (&cnt[0][0])[i] = 0u;
            __syncthreads();
            uint64_t key[kSegItems];
            uint32_t val[kSegItems];
#pragma unroll
            for (int k = 0; k < kSegItems; ++k) {
                const int idx = wbase + k * kWarp + lane;
                const bool ok = k < kn && idx < rem;
                key[k] = ok ? sk[c0 + idx] : 0ull;
                val[k] = ok ? sv[c0 + idx] : 0u;
            }
            uint32_t rnk[kSegItems];
            warp_rank(key, kn, wbase, rem, shift, mask, cnt[warp], rnk);
            __syncthreads();
            // per-warp prefix within the chunk (no digit starts: the
            // running offsets place the chunk)
            const int d = threadIdx.x;
            uint32_t run = 0;
#pragma unroll
            for (int w = 0; w < kSegWarps; ++w) {
                const uint32_t c = cnt[w][d];
                cnt[w][d] = run;
                run += c;
            }
            __syncthreads();
#pragma unroll
            for (int k = 0; k < kSegItems; ++k) {
                if (k >= kn) break;
                if (wbase + k * kWarp + lane < rem) {
                    const uint32_t dg = (uint32_t)(key[k] >> shift) & mask;
                    const uint32_t pos = off[dg] + cnt[warp][dg] + rnk[k];
                    dk[pos] = key[k];
                    dv[pos] = val[k];
                }
            }
            __syncthreads();
            off[d] += run;
        }
        __syncthreads();
        uint64_t* tk = sk; sk = dk; dk = tk;
        uint32_t* tv = sv; sv = dv; dv = tv;
        in_out = !in_out;
    }
    if (!in_out) {  // an even number of passes ran: copy into (kout, vout)
        for (uint32_t i = threadIdx.x; i < n; i += kSegThreads) {
            kout[b + i] = kin[b + i];
            vout[b + i] = vin[b + i];
        }
    }
}

// Blocks [0, nseg) sort one segment each when it holds more than 256 keys
// (and return at once otherwise); blocks nseg + g, g >= 0, give warp w the
// segment 8g + w when it holds 1 to 256 keys. The large segments come first
// in launch order so their longer sorts start early.
__global__ void __launch_bounds__(kSegThreads, 4)
k_seg_sort(uint64_t* kin, uint32_t* vin, uint64_t* kout, uint32_t* vout, const uint32_t* __restrict__ start,
           const uint32_t* __restrict__ num_keys, uint32_t cap, uint32_t nseg, int begin_bit) {
    // One buffer, carved two ways: the block paths' key / value / digit
    // count arrays, or each warp's padded staging slice (keys, values, sort
    // indices) for the warp path.
    constexpr int kPadCap = kWarpCap + kWarpCap / 8;
    constexpr int kWarpBytes = kPadCap * 8 + kWarpCap * 4 + kPadCap * 4;
    constexpr int kBlockBytes = kCtaCap * 8 + kCtaCap * 4 + kSegWarps * kLocalRadix * 4;
    constexpr int kRawBytes = kSegWarps * kWarpBytes > kBlockBytes ? kSegWarps * kWarpBytes : kBlockBytes;
    __shared__ __align__(16) unsigned char s_raw[kRawBytes];
    uint64_t* s_key = reinterpret_cast<uint64_t*>(s_raw);
    uint32_t* s_val = reinterpret_cast<uint32_t*>(s_raw + kCtaCap * 8);
    auto s_cnt = reinterpret_cast<uint32_t (*)[kLocalRadix]>(s_raw + kCtaCap * 12);
    __shared__ uint32_t s_off[kLocalRadix];
    __shared__ uint32_t s_red[2 * kSegWarps + 2];
    const int warp = threadIdx.x >> 5;
    pdl_wait();
    const uint32_t n_all = min(*num_keys, cap);
    // segment s as [b, e), clamped into [0, n]
    auto bounds = [&](uint32_t s, uint32_t& b, uint32_t& e) {
        e = min(__ldg(start + s + 1), n_all);
        b = min(__ldg(start + s), e);
    };
    if (blockIdx.x < nseg) {
        uint32_t b, e;
        bounds(blockIdx.x, b, e);
        const uint32_t n = e - b;
        if (n <= (uint32_t)kWarpCap) return;  // uniform over the block
        if (n <= (uint32_t)kCtaCap)
            block_sort_smem(kin, vin, kout, vout, b, (int)n, begin_bit, s_key, s_val, s_cnt, s_red);
        else
            block_sort_global(kin, vin, kout, vout, b, n, begin_bit, s_cnt, s_off, s_red);
        return;
    }
    const uint32_t s = (blockIdx.x - nseg) * kSegWarps + warp;
    if (s >= nseg) return;
    uint32_t b, e;
    bounds(s, b, e);
    const int n = (int)(e - b);
    if (n == 0 || n > kWarpCap) return;
    unsigned char* wraw = s_raw + warp * kWarpBytes;
    uint64_t* bk = reinterpret_cast<uint64_t*>(wraw);
    uint32_t* bv = reinterpret_cast<uint32_t*>(wraw + kPadCap * 8);
    uint32_t* bi = reinterpret_cast<uint32_t*>(wraw + kPadCap * 8 + kWarpCap * 4);
    if (n <= 32)
        warp_sort<1>(kin, vin, kout, vout, b, n, begin_bit, bk, bv, bi);
    else if (n <= 64)
        warp_sort<2>(kin, vin, kout, vout, b, n, begin_bit, bk, bv, bi);
    else if (n <= 128)
        warp_sort<4>(kin, vin, kout, vout, b, n, begin_bit, bk, bv, bi);
    else
        warp_sort<8>(kin, vin, kout, vout, b, n, begin_bit, bk, bv, bi);
}

// Scratch: [partition histograms, sized for 11-bit digits | segment starts].
size_t seg_start_offset_words(int64_t key_capacity) { return sort_scratch_bytes(key_capacity, 11) / 4; }

size_t seg_starts_words(int64_t key_capacity) {
    const size_t w = sort_scratch_bytes(key_capacity, 11) / 4;
    const size_t most = (size_t(1) << kMaxSegBits) + 1;
    return w < most ? w : most;
}

}  // namespace

size_t sort_segmented_scratch_bytes(int64_t key_capacity) {
    return (seg_start_offset_words(key_capacity) + seg_starts_words(key_capacity)) * sizeof(uint32_t);
}

bool sort_segmented_supported(int64_t key_capacity, int begin_bit, int end_bit) {
    if (begin_bit < 0 || begin_bit >= kSplitBit || end_bit <= kSplitBit || end_bit - kSplitBit > kMaxSegBits)
        return false;
    const uint64_t nseg = uint64_t(1) << (end_bit - kSplitBit);
    return nseg + 1 <= seg_starts_words(key_capacity);
}

int sort_segmented_first_digit(int end_bit, int digit_bits) {
    // Partition by the segment bits: as few passes as digits of at most
    // digit_bits bits allow, their width split evenly (13 segment bits at
    // digit_bits 8 or 9: 7 + 6); 4 bits at least.
    const int seg_bits = end_bit - kSplitBit;
    const int max_digit = digit_bits < 4 ? 4 : (digit_bits > 11 ? 11 : digit_bits);
    const int passes = (seg_bits + max_digit - 1) / max_digit;
    const int digit = (seg_bits + passes - 1) / passes;
    return digit < 4 ? 4 : digit;
}

cudaError_t launch_sort_segmented(const uint32_t* num_keys, int64_t key_capacity, int begin_bit, int end_bit,
                                  int digit_bits, uint64_t* keys, uint32_t* vals, uint64_t* keys_alt,
                                  uint32_t* vals_alt, void* scratch, int* in_alt, cudaStream_t stream,
                                  uint32_t* ranges, uint32_t ntiles, bool first_pass_done) {
    const int seg_bits = end_bit - kSplitBit;
    const int digit = sort_segmented_first_digit(end_bit, digit_bits);
    // With first_pass_done the keys already stand stably partitioned by the
    // first digit (the fused compaction): the passes start at the second.
    const int part_begin = first_pass_done ? kSplitBit + digit : kSplitBit;
    int part_alt = 0;
    cudaError_t e = cudaSuccess;
    if (part_begin < end_bit) {
        e = launch_sort(num_keys, key_capacity, part_begin, end_bit, digit, keys, vals, keys_alt, vals_alt, scratch,
                        &part_alt, stream);
        if (e != cudaSuccess) return e;
    }
    uint64_t* pk = part_alt ? keys_alt : keys;
    uint32_t* pv = part_alt ? vals_alt : vals;
    uint64_t* ok = part_alt ? keys : keys_alt;
    uint32_t* ov = part_alt ? vals : vals_alt;
    uint32_t* start = static_cast<uint32_t*>(scratch) + seg_start_offset_words(key_capacity);
    const uint32_t nseg = 1u << seg_bits;
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t spans = (key_capacity + 1 + 1023) / 1024;
    e = launch_pdl(k_seg_bounds, dim3((unsigned)(spans < sms * 8 ? spans : sms * 8)), dim3(256), 0, stream,
                   (const uint64_t*)pk, num_keys, (uint32_t)key_capacity, nseg - 1u, nseg, start,
                   reinterpret_cast<uint2*>(ranges), ntiles);
    if (e != cudaSuccess) return e;
    e = launch_pdl(k_seg_sort, dim3(nseg + (nseg + kSegWarps - 1) / kSegWarps), dim3(kSegThreads), 0, stream, pk, pv,
                   ok, ov, (const uint32_t*)start, num_keys, (uint32_t)key_capacity, nseg, begin_bit);
    if (e != cudaSuccess) return e;
    *in_alt = !part_alt;
    return cudaGetLastError();
}

}  // namespace ws
