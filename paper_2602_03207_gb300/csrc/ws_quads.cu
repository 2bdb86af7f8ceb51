// The paper's own render design (§3.3 sort stage, §3.4 rasterisation stage),
// re-expressed as CUDA for comparison with the tile path:
//   1. the visible splats are compacted and sorted by their 32-bit float
//      depth with four stable 8-bit passes (§3.3: full 32-bit sort, LSD,
//      each pass histogram / scan / scatter);
//   2. each splat is drawn as one quad sized by its opacity (E8:
//      r = sqrt(ln(255 sigma))) along its ellipse axes, carrying the local
//      coordinate p of E9 (p . p = q / 2, so the Gaussian is e^{-p.p});
//   3. the quads are composited back to front with "over" (§2.1) into an
//      FP32 image: C = a c + (1 - a) C.
// A graphics pipeline blends fragments in primitive order. Software must
// keep that order per pixel, so the quads are binned to screen tiles in depth
// order (emission in sorted order, then a stable partition by tile), and each
// tile composites its quads back to front. Per pixel the quad's fragment is
// the pixel centre inside |p_x|, |p_y| <= r; a = min(0.99, sigma e^{-p.p}), and
// fragments with a < 1/255 are skipped as in the tile path, so both
// paths produce the same image.
#include "ws_common.cuh"
#include "ws_kernels.cuh"

namespace ws {

namespace {

constexpr int kQuadThreads = 256;
constexpr int kQuadBatch = 256;

// Per-splat quad: p = M d maps a pixel offset d from the centre to the local
// coordinate; r is the E8 radius; the tile rectangle covers the quad's box.
struct QuadRec {
    float m00, m01, m10, m11;  // M (row-major)
    float r;                   // E8 cutoff radius in local units
    float hx, hy;              // half-widths of the quad's axis-aligned box (px)
    float pad;
};

// Quads of the visible splats (tiles_touched > 0). From the conic Q = Sigma'^{-1}
// with eigenpairs (mu_k, e_k): M = diag(sqrt(mu_1 / 2), sqrt(mu_2 / 2)) [e_1 e_2]^T,
// so p . p = d^T Q d / 2. The quad |p_x|, |p_y| <= r has corners
// d = sqrt(2) r (+-e_1 / sqrt(mu_1) +- e_2 / sqrt(mu_2)).
// Also writes the per-Gaussian items of the compaction: one "tile" (0) per
// visible splat, so the emission produces (depth bits, index) in index order.
__global__ void __launch_bounds__(kQuadThreads)
k_quad_setup(int64_t n, const float4* __restrict__ splats, const uint32_t* __restrict__ tiles_touched, const Frame f, QuadRec* __restrict__ quad,
             uint32_t* __restrict__ one, uint2* __restrict__ rect0) {
    pdl_wait();
    const int64_t i = (int64_t)blockIdx.x * kQuadThreads + threadIdx.x;
    if (i >= n) return;
    const bool vis = __ldg(tiles_touched + i) > 0u;
    one[i] = vis ? 1u : 0u;
    rect0[i] = make_uint2(0u, 0u);
    if (!vis) return;
    const float4 k4 = __ldg(splats + kSplatVec4 * i + 1);
    const float a = k4.x, b = k4.y, c = k4.z, sigma = k4.w;
    const float m = 0.5f * (a + c), h = 0.5f * (a - c);
    const float d = sqrtf(fmaf(h, h, b * b));
    const float mu2 = m + d;                         // larger eigenvalue: the minor axis
    const float mu1 = fmaf(a, c, -b * b) / mu2;      // smaller (det / mu2: no cancellation): the major axis
    // unit eigenvector of mu1 from the better-conditioned row of (Q - mu1 I)
    float ex = 1.f, ey = 0.f;
    if (d > 0.f) {
        if (h <= 0.f) {
            const float nn = hypotf(d - h, b);
            ex = (d - h) / nn;
            ey = -b / nn;
        } else {
            const float nn = hypotf(b, d + h);
            ex = -b / nn;
            ey = (d + h) / nn;
        }
    }
    const float s1 = sqrtf(0.5f * mu1), s2 = sqrtf(0.5f * mu2);
    QuadRec q;
    q.m00 = s1 * ex;
    q.m01 = s1 * ey;
    q.m10 = -s2 * ey;
    q.m11 = s2 * ex;
    const float lr = (f.flags & WS_CFG_FIXED_RADIUS) ? kLn255 : fmaxf(0.f, kLn255 + logf(sigma));
    q.r = sqrtf(lr);
    // corners: d = sqrt(2) r (+-e1 / sqrt(mu1) +- e2 / sqrt(mu2)), e2 = (-ey, ex);
    // a small margin keeps rounding from dropping a tile
    const float k1 = 1.41421356f * q.r * rsqrtf(mu1), k2 = 1.41421356f * q.r * rsqrtf(mu2);
    q.hx = (k1 * fabsf(ex) + k2 * fabsf(ey)) * 1.0001f + 1e-3f;
    q.hy = (k1 * fabsf(ey) + k2 * fabsf(ex)) * 1.0001f + 1e-3f;
    q.pad = 0.f;
    quad[i] = q;
}

// The binning items in depth order: item k (rank) is the k-th splat of the
// depth sort; its rectangle is the tiles of its quad's box, its depth 0, so
// the emission writes (tile << 31, rank) pairs in rank order.
__global__ void __launch_bounds__(kQuadThreads)
k_quad_bin_items(int64_t n, const uint32_t* __restrict__ num_vis, const uint32_t* __restrict__ order,
                 const float4* __restrict__ splats, const QuadRec* __restrict__ quad, const Frame f,
                 uint32_t* __restrict__ touched, uint2* __restrict__ rect, float* __restrict__ zero_depth) {
    pdl_wait();
    const int64_t k = (int64_t)blockIdx.x * kQuadThreads + threadIdx.x;
    if (k >= n) return;
    zero_depth[k] = 0.f;
    if (k >= (int64_t)*num_vis) {
        touched[k] = 0u;
        return;
    }
    const uint32_t g = __ldg(order + k);
    const float4 m = __ldg(splats + kSplatVec4 * g);
    const QuadRec q = quad[g];
    const float cx = m.x + m.z, cy = m.y + m.w;
    const float its = 1.f / (float)f.TS;
    const float lox = cx - q.hx, hix = cx + q.hx, loy = cy - q.hy, hiy = cy + q.hy;
    const bool on = hix >= 0.f && lox < (float)f.W && hiy >= 0.f && loy < (float)f.H;
    if (!on) {
        touched[k] = 0u;
        return;
    }
    const uint32_t x0 = (uint32_t)fminf((float)(f.TX - 1), fmaxf(0.f, floorf(lox * its)));
    const uint32_t x1 = (uint32_t)fminf((float)(f.TX - 1), fmaxf(0.f, floorf(hix * its)));
    const uint32_t y0 = (uint32_t)fminf((float)(f.TY - 1), fmaxf(0.f, floorf(loy * its)));
    const uint32_t y1 = (uint32_t)fminf((float)(f.TY - 1), fmaxf(0.f, floorf(hiy * its)));
    rect[k] = make_uint2(x0 | (y0 << 16), x1 | (y1 << 16));
    touched[k] = (x1 - x0 + 1) * (y1 - y0 + 1);
}

struct QuadStage {
    float cx, cy;          // tile-relative centre
    float m00, m01, m10, m11;
    float r, l2s;          // E8 radius, log2(sigma)
    float cr, cg, cb, pad;
};

// One block per tile, one thread per pixel (TS = 16: 256 pixels), the tile's
// quads back to front (highest rank first) in batches staged in shared
// memory; a warp skips a quad whose box misses its 8x4 pixel block.
template <int TS>
__global__ void __launch_bounds__(TS * TS >= 256 ? 256 : TS * TS)
k_blend_quads(const uint2* __restrict__ ranges, const uint32_t* __restrict__ ranks,
              const uint32_t* __restrict__ order, const float4* __restrict__ splats,
              const QuadRec* __restrict__ quad, const Frame f, float* __restrict__ image, float* __restrict__ t_final) {
    constexpr int THREADS = TS * TS >= 256 ? 256 : TS * TS;
    constexpr int WARPS = THREADS / 32;
    constexpr int PPT = TS * TS / THREADS;
    constexpr int BW = 8, BH = 4, BPR = TS / BW, BROWS = TS / BH;
    __shared__ QuadStage s_q[kQuadBatch];
    __shared__ uint32_t s_mask[kQuadBatch];
    pdl_wait();
    const int tile = blockIdx.x;
    const uint2 range = ranges[tile];
    const int tx = tile % f.TX, ty = tile / f.TX;
    const float ox = (float)(tx * TS), oy = (float)(ty * TS);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;

    float px[PPT], py[PPT], T[PPT], C0[PPT], C1[PPT], C2[PPT];
#pragma unroll
    for (int k = 0; k < PPT; ++k) {
        const int b = warp + k * WARPS;
        px[k] = (float)((b % BPR) * BW + (lane & 7)) + 0.5f;
        py[k] = (float)((b / BPR) * BH + (lane >> 3)) + 0.5f;
        T[k] = 1.f;
        C0[k] = f.bg[0];
        C1[k] = f.bg[1];
        C2[k] = f.bg[2];
    }
    for (int end = (int)(range.y - range.x); end > 0; end -= kQuadBatch) {
        const int lo = max(0, end - kQuadBatch);
        const int cnt = end - lo;
        __syncthreads();
        for (int j = threadIdx.x; j < cnt; j += THREADS) {
            const uint32_t g = __ldg(order + __ldg(ranks + range.x + lo + j));
            const float4 m = __ldg(splats + kSplatVec4 * g);
            const float op = __ldg(splats + kSplatVec4 * g + 1).w;
            const float4 cl = __ldg(splats + kSplatVec4 * g + 2);
            const QuadRec q = quad[g];
            QuadStage st;
            st.cx = __fadd_rn(__fsub_rn(m.x, ox), m.z);
            st.cy = __fadd_rn(__fsub_rn(m.y, oy), m.w);
            st.m00 = q.m00;
            st.m01 = q.m01;
            st.m10 = q.m10;
            st.m11 = q.m11;
            st.r = q.r;
            st.l2s = log2f(op);
            st.cr = cl.x;
            st.cg = cl.y;
            st.cb = cl.z;
            st.pad = 0.f;
            s_q[j] = st;
            s_mask[j] = box_block_mask<BW, BH, BPR, BROWS>(st.cx - q.hx, st.cx + q.hx, st.cy - q.hy, st.cy + q.hy);
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < PPT; ++k) {
            const int blk = warp + k * WARPS;
            for (int base = ((cnt - 1) >> 5) << 5; base >= 0; base -= 32) {
                const int jj = base + lane;
                uint32_t bits = __ballot_sync(kFull, jj < cnt && ((s_mask[jj] >> blk) & 1u));
                while (bits) {  // back to front: highest position first
                    const int hb = 31 - __clz(bits);
                    bits &= ~(1u << hb);
                    const QuadStage& st = s_q[base + hb];
                    const float dx = px[k] - st.cx, dy = py[k] - st.cy;
                    // E9: local coordinate, a = p . p, fragment inside the quad
                    const float p0 = fmaf(st.m00, dx, st.m01 * dy), p1 = fmaf(st.m10, dx, st.m11 * dy);
                    const float a = fmaf(p0, p0, p1 * p1);
                    const bool inside = fabsf(p0) <= st.r && fabsf(p1) <= st.r;
                    const float e = fmaf(-kLog2e, a, st.l2s);  // log2(sigma e^{-a})
                    const bool keep = inside && e >= kLog2AlphaMin;
                    const float alpha = keep ? fminf(kAlphaMax, ex2_approx(e)) : 0.f;
                    // "over": C = a c + (1 - a) C
                    C0[k] = fmaf(alpha, st.cr - C0[k], C0[k]);
                    C1[k] = fmaf(alpha, st.cg - C1[k], C1[k]);
                    C2[k] = fmaf(alpha, st.cb - C2[k], C2[k]);
                    T[k] = T[k] - alpha * T[k];
                }
            }
        }
    }
#pragma unroll
    for (int k = 0; k < PPT; ++k) {
        const int gx = tx * TS + (int)px[k], gy = ty * TS + (int)py[k];
        if (gx < f.W && gy < f.H) {
            const size_t pix = (size_t)gy * f.W + gx;
            image[3 * pix] = C0[k];
            image[3 * pix + 1] = C1[k];
            image[3 * pix + 2] = C2[k];
            t_final[pix] = T[k];
        }
    }
}

size_t align256(size_t v) { return (v + 255) & ~size_t(255); }

}  // namespace

QuadLayout quad_layout(int64_t n, int64_t key_capacity, int64_t ntiles) {
    QuadLayout L;
    const size_t n1 = (size_t)(n > 0 ? n : 1);
    const int64_t sort_keys = n > key_capacity ? n : key_capacity;
    size_t off = align256(kStatusBytes);
    L.sort = off;
    off += align256(sort_scratch_bytes(sort_keys, 11));
    L.cull = off;
    off += align256(cull_scratch_bytes(n));
    L.dkeys = off;      off += align256(n1 * 8);
    L.dkeys_alt = off;  off += align256(n1 * 8);
    L.dvals = off;      off += align256(n1 * 4);
    L.dvals_alt = off;  off += align256(n1 * 4);
    L.offsets = off;    off += align256((n1 + 1) * 4);
    L.quad = off;       off += align256(n1 * sizeof(QuadRec));
    L.one = off;        off += align256(n1 * 4);
    L.rect = off;       off += align256(n1 * 8);
    L.zdepth = off;     off += align256(n1 * 4);
    L.num_vis = off;    off += 256;
    L.ranges = off;     off += align256((size_t)(ntiles > 0 ? ntiles : 1) * 8);
    L.total = off;
    return L;
}

cudaError_t launch_render_quads(int64_t n, const float* splats, const float* depth, const uint32_t* tiles_touched,
                                const Frame& f, int64_t key_capacity, uint64_t* keys, uint32_t* vals,
                                uint64_t* keys_alt, uint32_t* vals_alt, uint32_t* num_keys, float* image,
                                float* t_final, void* workspace, cudaStream_t stream) {
    const int64_t ntiles = (int64_t)f.TX * f.TY;
    const QuadLayout L = quad_layout(n, key_capacity, ntiles);
    char* w = static_cast<char*>(workspace);
    uint32_t* status = reinterpret_cast<uint32_t*>(w);
    uint64_t* dkeys = reinterpret_cast<uint64_t*>(w + L.dkeys);
    uint64_t* dkeys_alt = reinterpret_cast<uint64_t*>(w + L.dkeys_alt);
    uint32_t* dvals = reinterpret_cast<uint32_t*>(w + L.dvals);
    uint32_t* dvals_alt = reinterpret_cast<uint32_t*>(w + L.dvals_alt);
    uint32_t* offsets = reinterpret_cast<uint32_t*>(w + L.offsets);
    QuadRec* quad = reinterpret_cast<QuadRec*>(w + L.quad);
    uint32_t* one = reinterpret_cast<uint32_t*>(w + L.one);
    uint2* rect = reinterpret_cast<uint2*>(w + L.rect);
    float* zdepth = reinterpret_cast<float*>(w + L.zdepth);
    uint32_t* num_vis = reinterpret_cast<uint32_t*>(w + L.num_vis);
    uint2* ranges = reinterpret_cast<uint2*>(w + L.ranges);
    const float4* s4 = reinterpret_cast<const float4*>(splats);
    const dim3 grid_n((unsigned)((n + kQuadThreads - 1) / kQuadThreads > 0 ? (n + kQuadThreads - 1) / kQuadThreads
                                                                               : 1));
    cudaError_t e;
    // 1. quads, and the compaction of the visible splats into (depth, index)
    if (n > 0) {
        e = launch_pdl(k_quad_setup, grid_n, dim3(kQuadThreads), 0, stream, n, s4, tiles_touched, f, quad, one,
                       rect);
        if (e != cudaSuccess) return e;
    }
    e = launch_cull(n, one, reinterpret_cast<const uint16_t*>(rect), depth, f, offsets, dkeys, dvals, n, num_vis,
                    status, w + L.cull, stream);
    if (e != cudaSuccess) return e;
    // 2. the 32-bit depth sort: four stable 8-bit passes (even: ends in dkeys)
    int in_alt = 0;
    e = launch_sort(num_vis, n, 0, 32, 8, dkeys, dvals, dkeys_alt, dvals_alt, w + L.sort, &in_alt, stream);
    if (e != cudaSuccess) return e;
    const uint32_t* order = in_alt ? dvals_alt : dvals;
    // 3. binning in depth order, then a stable partition by tile
    if (n > 0) {
        e = launch_pdl(k_quad_bin_items, grid_n, dim3(kQuadThreads), 0, stream, n, (const uint32_t*)num_vis, order,
                       s4, (const QuadRec*)quad, f, one, rect, zdepth);
        if (e != cudaSuccess) return e;
    }
    e = launch_cull(n, one, reinterpret_cast<const uint16_t*>(rect), zdepth, f, offsets, keys, vals, key_capacity,
                    num_keys, status, w + L.cull, stream);
    if (e != cudaSuccess) return e;
    int tile_bits = 1;
    while ((int64_t(1) << tile_bits) < ntiles) ++tile_bits;
    int part_alt = 0;
    e = launch_sort(num_keys, key_capacity, 31, 31 + tile_bits, 7, keys, vals, keys_alt, vals_alt, w + L.sort,
                    &part_alt, stream);
    if (e != cudaSuccess) return e;
    const uint64_t* pk = part_alt ? keys_alt : keys;
    const uint32_t* pv = part_alt ? vals_alt : vals;
    e = launch_tile_ranges(pk, num_keys, reinterpret_cast<uint32_t*>(ranges), (uint32_t)ntiles, 0u, stream);
    if (e != cudaSuccess) return e;
    // 4. back-to-front quads per tile
    switch (f.TS) {
        case 8:
            return launch_pdl(k_blend_quads<8>, dim3((unsigned)ntiles), dim3(64), 0, stream, (const uint2*)ranges, pv,
                              order, s4, (const QuadRec*)quad, f, image, t_final);
        case 16:
            return launch_pdl(k_blend_quads<16>, dim3((unsigned)ntiles), dim3(256), 0, stream, (const uint2*)ranges,
                              pv, order, s4, (const QuadRec*)quad, f, image, t_final);
        case 32:
            return launch_pdl(k_blend_quads<32>, dim3((unsigned)ntiles), dim3(256), 0, stream, (const uint2*)ranges,
                              pv, order, s4, (const QuadRec*)quad, f, image, t_final);
        default:
            return cudaErrorInvalidValue;
    }
}

}  // namespace ws
