// Pre-processing stage (paper §3.2 with the covariance/colour model of §2.1
// and the opacity culling and opacity-aware extent of §3.4).
//
// One thread per Gaussian, 128-thread blocks. HBM-bound: 236 B of input per
// visible Gaussian (59 floats), 16 B per opacity-culled one (logit, centre),
// 44 B per one culled later (no SH); 64 B of output each (the 48-byte splat
// record, depth, rect, tile count). The 192-byte SH
// record is the bulk of the traffic; each warp copies the SH of its
// Gaussians that will probably be visible into shared memory with
// asynchronous, coalesced 16-byte copies issued before the projection math
// (a per-thread load of a 192-byte stride would touch 32 cache lines per
// instruction), padded to 52 floats so the per-lane float4 reads are
// bank-conflict free.
#include "ws_common.cuh"
#include "ws_kernels.cuh"
#include "ws_project.cuh"

namespace ws {

namespace {

constexpr int kPreThreads = 128;

__global__ void __launch_bounds__(kPreThreads)
k_preprocess(int64_t n, const float* __restrict__ means, const float* __restrict__ log_scales,
             const float4* __restrict__ quats, const float* __restrict__ logits,
             const float4* __restrict__ sh, const Frame f, float4* __restrict__ splats,
             float* __restrict__ depth, uint2* __restrict__ rect, uint32_t* __restrict__ tiles_touched) {
    __shared__ __align__(16) float s_sh[kPreThreads / kWarp][kWarp * kShPad];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t i = (int64_t)blockIdx.x * kPreThreads + threadIdx.x;
    const bool valid = i < n;
    const int64_t warp_first = (int64_t)blockIdx.x * kPreThreads + warp * kWarp;
    pdl_wait();

    // All per-Gaussian inputs but the SH are requested at once.
    float logit = 0.f, x = 0.f, y = 0.f, z = 0.f, l0 = 0.f, l1 = 0.f, l2 = 0.f;
    float4 q = make_float4(0.f, 0.f, 0.f, 0.f);
    if (valid) {
        logit = __ldg(logits + i);
        x = __ldg(means + 3 * i);
        y = __ldg(means + 3 * i + 1);
        z = __ldg(means + 3 * i + 2);
        q = __ldg(quats + i);
        l0 = __ldg(log_scales + 3 * i);
        l1 = __ldg(log_scales + 3 * i + 1);
        l2 = __ldg(log_scales + 3 * i + 2);
    }
    const bool opaque_enough = valid && passes_opacity(f, logit);
    const float d = valid ? view_depth(f, x, y, z) : 0.f;
    // Stage the SH records of the lanes that will probably be visible into
    // shared memory asynchronously (16-byte copies, coalesced across the
    // warp), so the copies overlap the projection below; lanes that turn out
    // visible without the hint get their record afterwards.
    const bool likely = opaque_enough && likely_visible(f, x, y, z, d, l0, l1, l2);
    const uint32_t need = __ballot_sync(kFull, likely);
    float* stage = s_sh[warp];
    const float4* src = sh + warp_first * 12;
    if (need) {
#pragma unroll
        for (int r = 0; r < 12; ++r) {
            const int vv = lane + r * kWarp;
            const int g = vv / 12, c = vv - g * 12;
            if ((need >> g) & 1u) cp_async16(stage + g * kShPad + 4 * c, src + vv);
        }
        asm volatile("cp.async.commit_group;" ::: "memory");
    }

    bool vis = false;
    Projection P;
    if (valid) {
        depth[i] = d;
        vis = opaque_enough && d > f.znear;
        if (vis) vis = project_splat(f, x, y, z, q, l0, l1, l2, logit, P);
    }
    const uint32_t late = __ballot_sync(kFull, vis && !likely);
    if (late) {
#pragma unroll
        for (int r = 0; r < 12; ++r) {
            const int vv = lane + r * kWarp;
            const int g = vv / 12, c = vv - g * 12;
            if ((late >> g) & 1u) cp_async16(stage + g * kShPad + 4 * c, src + vv);
        }
        asm volatile("cp.async.commit_group;" ::: "memory");
    }

    // SH colour (§2.1, §3.2) for the visible lanes from the staged records.
    float3 c3 = make_float3(0.f, 0.f, 0.f);
    if (need | late) {
        asm volatile("cp.async.wait_group 0;" ::: "memory");
        __syncwarp();
        if (vis) {
            const float dx = x - f.campos[0], dy = y - f.campos[1], dz = z - f.campos[2];
            const float inv = rsqrtf(dx * dx + dy * dy + dz * dz);
            sh_eval(dx * inv, dy * inv, dz * inv, stage + lane * kShPad, c3);
        }
    }
    // Every lane stores its entries (zeros for a culled Gaussian), so the
    // warp writes whole 32-byte sectors: a sector left partly written would
    // cost a read of it from DRAM when it leaves the L2.
    if (valid) {
        store_splat(splats + kSplatVec4 * i, vis, P, c3);
        rect[i] = vis ? make_uint2(P.x0 | (P.y0 << 16), P.x1 | (P.y1 << 16)) : make_uint2(0u, 0u);
        tiles_touched[i] = vis ? (P.x1 - P.x0 + 1) * (P.y1 - P.y0 + 1) : 0u;
    }
}

}  // namespace

cudaError_t launch_preprocess(int64_t n, const float* means, const float* log_scales,
                              const float* quats, const float* logits, const float* sh,
                              const Frame& f, float* splats, float* depth, uint16_t* rect,
                              uint32_t* tiles_touched, cudaStream_t stream) {
    if (n == 0) return cudaSuccess;
    const int64_t blocks = (n + kPreThreads - 1) / kPreThreads;
    return launch_pdl(k_preprocess, dim3((unsigned)blocks), dim3(kPreThreads), 0, stream, n, means, log_scales,
                      reinterpret_cast<const float4*>(quats), logits, reinterpret_cast<const float4*>(sh), f,
                      reinterpret_cast<float4*>(splats), depth, reinterpret_cast<uint2*>(rect), tiles_touched);
}

}  // namespace ws
