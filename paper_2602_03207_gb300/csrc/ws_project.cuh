// Per-Gaussian device arithmetic of the pre-processing stage (paper §3.2,
// §2.1, §3.4), shared by the single-view and the batched kernels so both
// produce bit-identical results for the same camera.
#pragma once

#include "ws_common.cuh"

namespace ws {

// Real SH basis of degree 3 (Condon-Shortley phase, index l*l + l + m) as
// homogeneous polynomials of the unit direction; constants are
// sqrt((2l+1)/(4 pi) (l-|m|)!/(l+|m|)!) times the polynomial's own factor.
__device__ __forceinline__ void sh_eval(float x, float y, float z, const float* kf, float3& out) {
    const float c0 = 0.28209479177387814f;
    const float c1 = 0.4886025119029199f;
    const float c2a = 1.0925484305920792f, c2b = 0.31539156525252005f, c2c = 0.5462742152960396f;
    const float c3a = 0.5900435899266435f, c3b = 2.890611442640554f, c3c = 0.4570457994644658f;
    const float c3d = 0.3731763325901154f, c3e = 1.445305721320277f;
    float xx = x * x, yy = y * y, zz = z * z;
    float b[16];
    b[0] = c0;
    b[1] = -c1 * y;
    b[2] = c1 * z;
    b[3] = -c1 * x;
    b[4] = c2a * x * y;
    b[5] = -c2a * y * z;
    b[6] = c2b * (2.f * zz - xx - yy);
    b[7] = -c2a * x * z;
    b[8] = c2c * (xx - yy);
    b[9] = -c3a * y * (3.f * xx - yy);
    b[10] = c3b * x * y * z;
    b[11] = -c3c * y * (4.f * zz - xx - yy);
    b[12] = c3d * z * (2.f * zz - 3.f * xx - 3.f * yy);
    b[13] = -c3c * x * (4.f * zz - xx - yy);
    b[14] = c3e * z * (xx - yy);
    b[15] = -c3a * x * (xx - 3.f * yy);
    // kf: 48 floats, coefficient-major [16][3], 16-byte aligned; read as
    // float4 (conflict-free from the padded shared-memory records).
    float k[48];
#pragma unroll
    for (int r4 = 0; r4 < 12; ++r4) {
        const float4 t = reinterpret_cast<const float4*>(kf)[r4];
        k[4 * r4] = t.x;
        k[4 * r4 + 1] = t.y;
        k[4 * r4 + 2] = t.z;
        k[4 * r4 + 3] = t.w;
    }
    float r = 0.5f, g = 0.5f, bl = 0.5f;
#pragma unroll
    for (int i = 0; i < 16; ++i) {
        r = fmaf(b[i], k[3 * i + 0], r);
        g = fmaf(b[i], k[3 * i + 1], g);
        bl = fmaf(b[i], k[3 * i + 2], bl);
    }
    out = make_float3(fmaxf(r, 0.f), fmaxf(g, 0.f), fmaxf(bl, 0.f));
}

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
    const uint32_t sa = (uint32_t)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(sa), "l"(gmem) : "memory");
}

// §3.2: the float32 view depth, each operation rounded in a fixed order.
__device__ __forceinline__ float view_depth(const Frame& f, float x, float y, float z) {
    return __fadd_rn(__fadd_rn(__fadd_rn(__fmul_rn(f.R[6], x), __fmul_rn(f.R[7], y)), __fmul_rn(f.R[8], z)),
                     f.t[2]);
}

// Whether a Gaussian in front of the near plane (depth d) will probably be
// visible: its projected centre inside the viewport widened by a bound on its
// screen extent, sqrt(2 ln 255) * 1.6 * f * max scale / d plus the dilation
// (1.6 covers the row norm of the Jacobian with the guard-band clamp). Only a
// prefetch hint: callers still handle a visible splat it missed.
__device__ __forceinline__ bool likely_visible(const Frame& f, float x, float y, float z, float d, float l0,
                                               float l1, float l2) {
    if (!(d > f.znear)) return false;
    const float cxs = __fmaf_rn(f.R[0], x, __fmaf_rn(f.R[1], y, __fmaf_rn(f.R[2], z, f.t[0])));
    const float cys = __fmaf_rn(f.R[3], x, __fmaf_rn(f.R[4], y, __fmaf_rn(f.R[5], z, f.t[1])));
    const float rd = 1.f / d;
    const float u = __fmaf_rn(f.fx * rd, cxs, f.cx), v = __fmaf_rn(f.fy * rd, cys, f.cy);
    const float smax = expf(fmaxf(l0, fmaxf(l1, l2)));
    const float m = 3.33f * (1.6f * fmaxf(f.fx, f.fy) * smax * rd + 0.6f) + 2.f;
    return u > -m && u < (float)f.W + m && v > -m && v < (float)f.H + m;
}

// §3.4 opacity culling: sigma < 1/255 <=> logit < -ln 254, decided exactly.
__device__ __forceinline__ bool passes_opacity(const Frame& f, float logit) {
    return (double)logit >= kOpacityLogitMin || (f.flags & WS_CFG_NO_OPACITY_CULL);
}

struct Projection {
    float4 m4;         // projected centre as double-float (x_hi, y_hi, x_lo, y_lo)
    float ca, cb, cc;  // conic = Sigma'^{-1}
    float sigma;       // peak opacity
    float t;           // tan(theta / 2), theta in [-pi/2, pi/2] the angle of Sigma''s major axis
    uint32_t x0, y0, x1, y1;  // tile rectangle (inclusive)
};

// t = tan(theta / 2) of the major axis of [[sxx, sxy], [sxy, syy]]: an
// eigenvector e from whichever row of (Sigma' - l1 I) is better conditioned,
// (d + h, sxy) or (sxy, d - h) with h = (sxx - syy) / 2, d = sqrt(h^2 +
// sxy^2), whose norm is sqrt(2 d (d + |h|)) either way; turned to e.x >= 0,
// t = e.y / (|e| + e.x). 0 for a circle. Any t within a few ulp will do: the
// record stores it and every user rebuilds the basis from the stored value.
__device__ __forceinline__ float major_axis_t(float sxx, float sxy, float syy) {
    const float h = 0.5f * (sxx - syy);
    const float d = sqrtf(fmaf(h, h, sxy * sxy));
    if (!(d > 0.f)) return 0.f;
    const float dh = d + fabsf(h);
    float ex = h >= 0.f ? dh : sxy;
    float ey = h >= 0.f ? sxy : dh;
    if (ex < 0.f) {
        ex = -ex;
        ey = -ey;
    }
    return __fdividef(ey, sqrtf(2.f * d * dh) + ex);
}

// Stores the splat record of one Gaussian (zeros when it is not visible).
__device__ __forceinline__ void store_splat(float4* __restrict__ dst, bool vis, const Projection& P, float3 c3) {
    const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
    dst[0] = vis ? P.m4 : z;
    dst[1] = vis ? make_float4(P.ca, P.cb, P.cc, P.sigma) : z;
    dst[2] = make_float4(c3.x, c3.y, c3.z, vis ? P.t : 0.f);
}

// det(Sigma') for Sigma' = V V^T + dilation I (rows V0, V1 of V; sxx, syy the
// diagonal with the dilation): by Lagrange's identity det(V V^T) =
// |V0 x V1|^2, so det(Sigma') = |V0 x V1|^2 + dilation (sxx + syy) -
// dilation^2, with sxx + syy - dilation = |V0|^2 + |V1|^2 + dilation: a sum
// of non-negative terms. sxx syy - sxy^2 would cancel for an elongated splat
// (condition number 3e4 costs it ~3e-4 of relative error in float32) and
// the conic, a common factor 1/det, would carry that error into every alpha.
__device__ __forceinline__ float sigma2d_det(const float V0[3], const float V1[3], float sxx, float syy, float dil) {
    const float c0 = fmaf(V0[1], V1[2], -V0[2] * V1[1]);
    const float c1 = fmaf(V0[2], V1[0], -V0[0] * V1[2]);
    const float c2 = fmaf(V0[0], V1[1], -V0[1] * V1[0]);
    const float cross2 = fmaf(c0, c0, fmaf(c1, c1, c2 * c2));
    return fmaf(dil, sxx + syy - dil, cross2);
}

// Projection of one Gaussian that passed the opacity and near-plane tests:
// Sigma = M M^T with M = R(q) diag(exp(log_scale)) (§2.1); the centre through
// the pinhole in double-float; Sigma' = V V^T + dilation I with V = J W M
// (EWA Jacobian J with the guard-band clamp) returned in sxx, sxy, syy;
// conic = Sigma'^{-1}. Returns false when the quaternion is zero or Sigma' is
// degenerate.
__device__ __forceinline__ bool project_core(const Frame& f, float x, float y, float z, float4 q, float l0, float l1,
                                             float l2, Projection& P, float& sxx, float& sxy, float& syy) {
    const float qn2 = q.x * q.x + q.y * q.y + q.z * q.z + q.w * q.w;
    if (qn2 == 0.f) return false;
    const float inv = rsqrtf(qn2);
    const float w = q.x * inv, qx = q.y * inv, qy = q.z * inv, qz = q.w * inv;
    const float R[9] = {1.f - 2.f * (qy * qy + qz * qz), 2.f * (qx * qy - w * qz), 2.f * (qx * qz + w * qy),
                        2.f * (qx * qy + w * qz), 1.f - 2.f * (qx * qx + qz * qz), 2.f * (qy * qz - w * qx),
                        2.f * (qx * qz - w * qy), 2.f * (qy * qz + w * qx), 1.f - 2.f * (qx * qx + qy * qy)};
    const float s0 = expf(l0), s1 = expf(l1), s2 = expf(l2);
    const float M[9] = {R[0] * s0, R[1] * s1, R[2] * s2, R[3] * s0, R[4] * s1,
                        R[5] * s2, R[6] * s0, R[7] * s1, R[8] * s2};
    // Camera-space centre in double-float, then the projected centre.
    const DF tx = df_affine3(f.R[0], f.R[1], f.R[2], x, y, z, f.t[0]);
    const DF ty = df_affine3(f.R[3], f.R[4], f.R[5], x, y, z, f.t[1]);
    const DF tz = df_affine3(f.R[6], f.R[7], f.R[8], x, y, z, f.t[2]);
    const DF mx = df_scale_add(f.fx, df_div(tx, tz), f.cx);
    const DF my = df_scale_add(f.fy, df_div(ty, tz), f.cy);
    P.m4 = make_float4(mx.hi, my.hi, mx.lo, my.lo);
    // EWA Jacobian with the guard-band clamp, T = J W.
    const float rz = 1.f / tz.hi;
    const float rx = fminf(f.limx, fmaxf(-f.limx, tx.hi * rz));
    const float ry = fminf(f.limy, fmaxf(-f.limy, ty.hi * rz));
    const float j00 = f.fx * rz, j02 = -f.fx * rx * rz, j11 = f.fy * rz, j12 = -f.fy * ry * rz;
    const float T0[3] = {j00 * f.R[0] + j02 * f.R[6], j00 * f.R[1] + j02 * f.R[7], j00 * f.R[2] + j02 * f.R[8]};
    const float T1[3] = {j11 * f.R[3] + j12 * f.R[6], j11 * f.R[4] + j12 * f.R[7], j11 * f.R[5] + j12 * f.R[8]};
    // V = T M (2x3); Sigma' = T Sigma T^T + dilation I = V V^T + dilation I:
    // sums of squares on the diagonal, no cancellation.
    float V0[3], V1[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        V0[k] = T0[0] * M[k] + T0[1] * M[3 + k] + T0[2] * M[6 + k];
        V1[k] = T1[0] * M[k] + T1[1] * M[3 + k] + T1[2] * M[6 + k];
    }
    sxx = V0[0] * V0[0] + V0[1] * V0[1] + V0[2] * V0[2] + f.dilation;
    sxy = V0[0] * V1[0] + V0[1] * V1[1] + V0[2] * V1[2];
    syy = V1[0] * V1[0] + V1[1] * V1[1] + V1[2] * V1[2] + f.dilation;
    const float det = sigma2d_det(V0, V1, sxx, syy, f.dilation);
    if (!(det > 0.f)) return false;
    const float id = 1.f / det;
    P.ca = syy * id;
    P.cb = -sxy * id;
    P.cc = sxx * id;
    P.t = major_axis_t(sxx, sxy, syy);
    return true;
}

// Viewport AABB test (§3.2) of the box [m - e, m + e] (the centre m as
// double-float hi + lo) and its tile rectangle. Returns false when the box
// misses the viewport (unless WS_CFG_NO_AABB_CULL keeps it, clamped).
__device__ __forceinline__ bool splat_rect(const Frame& f, float mxh, float mxl, float myh, float myl, float ex,
                                           float ey, Projection& P) {
    const float lox = __fadd_rn(__fsub_rn(mxh, ex), mxl), hix = __fadd_rn(__fadd_rn(mxh, ex), mxl);
    const float loy = __fadd_rn(__fsub_rn(myh, ey), myl), hiy = __fadd_rn(__fadd_rn(myh, ey), myl);
    const bool on = hix >= 0.f && lox < (float)f.W && hiy >= 0.f && loy < (float)f.H;
    if (!on && !(f.flags & WS_CFG_NO_AABB_CULL)) return false;
    const float its = 1.f / (float)f.TS;  // exact: TS is a power of two
    P.x0 = (uint32_t)fminf((float)(f.TX - 1), fmaxf(0.f, floorf(lox * its)));
    P.x1 = (uint32_t)fminf((float)(f.TX - 1), fmaxf(0.f, floorf(hix * its)));
    P.y0 = (uint32_t)fminf((float)(f.TY - 1), fmaxf(0.f, floorf(loy * its)));
    P.y1 = (uint32_t)fminf((float)(f.TY - 1), fmaxf(0.f, floorf(hiy * its)));
    return true;
}

// project_core, then sigma and the opacity-aware extent
// e = sqrt(2 ln(255 sigma) diag Sigma') (§3.4) and splat_rect.
__device__ __forceinline__ bool project_splat(const Frame& f, float x, float y, float z, float4 q, float l0,
                                              float l1, float l2, float logit, Projection& P) {
    float sxx, sxy, syy;
    if (!project_core(f, x, y, z, q, l0, l1, l2, P, sxx, sxy, syy)) return false;
    // sigma and the opacity-aware extent (§3.4): q_c = 2 ln(255 sigma)
    const float en = expf(-logit);
    P.sigma = 1.f / (1.f + en);
    // WS_CFG_FIXED_RADIUS (ablation): the box every splat would need at
    // sigma = 1, independent of its opacity (conservative, only larger).
    const float qc = (f.flags & WS_CFG_FIXED_RADIUS) ? 2.f * kLn255 : fmaxf(0.f, 2.f * (kLn255 - log1pf(en)));
    const float ex = sqrtf(qc * sxx), ey = sqrtf(qc * syy);
    return splat_rect(f, P.m4.x, P.m4.z, P.m4.y, P.m4.w, ex, ey, P);
}

// SH records staged in shared memory are padded to 52 floats so per-lane
// float4 reads of 32 consecutive records are bank-conflict free.
constexpr int kShPad = 52;

// Real SH basis of degree 3 (Condon-Shortley phase, index l*l + l + m) and
// its gradient with respect to the (unit) direction.
__device__ __forceinline__ void sh_basis_grad(float x, float y, float z, float* Y, float (*dY)[3]) {
    const float k0 = 0.28209479177387814f, k1 = 0.4886025119029199f;
    const float k2a = 1.0925484305920792f, k2b = 0.31539156525252005f, k2c = 0.5462742152960396f;
    const float k3a = 0.5900435899266435f, k3b = 2.890611442640554f, k3c = 0.4570457994644658f;
    const float k3d = 0.3731763325901154f, k3e = 1.445305721320277f;
    const float xx = x * x, yy = y * y, zz = z * z;
    Y[0] = k0;
    dY[0][0] = dY[0][1] = dY[0][2] = 0.f;
    Y[1] = -k1 * y;  dY[1][0] = 0.f; dY[1][1] = -k1; dY[1][2] = 0.f;
    Y[2] = k1 * z;   dY[2][0] = 0.f; dY[2][1] = 0.f; dY[2][2] = k1;
    Y[3] = -k1 * x;  dY[3][0] = -k1; dY[3][1] = 0.f; dY[3][2] = 0.f;
    Y[4] = k2a * x * y;  dY[4][0] = k2a * y; dY[4][1] = k2a * x; dY[4][2] = 0.f;
    Y[5] = -k2a * y * z; dY[5][0] = 0.f; dY[5][1] = -k2a * z; dY[5][2] = -k2a * y;
    Y[6] = k2b * (2.f * zz - xx - yy);
    dY[6][0] = -2.f * k2b * x; dY[6][1] = -2.f * k2b * y; dY[6][2] = 4.f * k2b * z;
    Y[7] = -k2a * x * z; dY[7][0] = -k2a * z; dY[7][1] = 0.f; dY[7][2] = -k2a * x;
    Y[8] = k2c * (xx - yy); dY[8][0] = 2.f * k2c * x; dY[8][1] = -2.f * k2c * y; dY[8][2] = 0.f;
    Y[9] = -k3a * y * (3.f * xx - yy);
    dY[9][0] = -6.f * k3a * x * y; dY[9][1] = -3.f * k3a * (xx - yy); dY[9][2] = 0.f;
    Y[10] = k3b * x * y * z;
    dY[10][0] = k3b * y * z; dY[10][1] = k3b * x * z; dY[10][2] = k3b * x * y;
    Y[11] = -k3c * y * (4.f * zz - xx - yy);
    dY[11][0] = 2.f * k3c * x * y; dY[11][1] = -k3c * (4.f * zz - xx - 3.f * yy); dY[11][2] = -8.f * k3c * y * z;
    Y[12] = k3d * z * (2.f * zz - 3.f * xx - 3.f * yy);
    dY[12][0] = -6.f * k3d * x * z; dY[12][1] = -6.f * k3d * y * z; dY[12][2] = k3d * (6.f * zz - 3.f * xx - 3.f * yy);
    Y[13] = -k3c * x * (4.f * zz - xx - yy);
    dY[13][0] = -k3c * (4.f * zz - 3.f * xx - yy); dY[13][1] = 2.f * k3c * x * y; dY[13][2] = -8.f * k3c * x * z;
    Y[14] = k3e * z * (xx - yy);
    dY[14][0] = 2.f * k3e * x * z; dY[14][1] = -2.f * k3e * y * z; dY[14][2] = k3e * (xx - yy);
    Y[15] = -k3a * x * (xx - 3.f * yy);
    dY[15][0] = -3.f * k3a * (xx - yy); dY[15][1] = 6.f * k3a * x * y; dY[15][2] = 0.f;
}


// Adjoint of project_splat's geometry for one view: given the summed pair
// derivatives pr[0..1] = dL/d(centre x, y) and pr[2..4] = dL/d(alpha, beta,
// gamma), the conic in the splat's axis basis (axis_basis(axis_t): q = alpha u^2 +
// 2 beta u v + gamma v^2 with u = e1 . d, v = e2 . d), ADDS dL/dmeans,
// dL/dlog_scales and dL/dquats into gm, gls, gq. The chain: conic =
// Sigma'^{-1}, Sigma' = V V^T + dilation I, V = J W M (the guard-band clamp of
// J passes no gradient), M = R(q) diag(exp(log_scale)), q normalised, and the
// pinhole projection of the centre.
//
// Why the axis basis: for an elongated splat (Sigma' eigenvalues 1e4 and 0.3
// px^2, say) the pixels far along its major axis give conic derivatives of
// order dp u^2 ~ 1e6 dp, while dL/dSigma' = -C dL/dC C scales the along-axis
// part by the conic's small eigenvalue squared (1e-8). In x, y coordinates
// that part is lost under the rounding of the large entries, and the
// gradient of the major axis's scale comes out wrong by several times its
// size; summed and transformed in the axis basis, each part keeps its own
// relative precision.
__device__ __forceinline__ void splat_adjoint(const Frame& f, const float X[3], float4 q4, const float ls[3],
                                              const float pr[9], float axis_t, float gm[3], float gls[3], float gq[4]) {
    // forward quantities
    const float qn2 = q4.x * q4.x + q4.y * q4.y + q4.z * q4.z + q4.w * q4.w;
    const float qinv = rsqrtf(qn2);
    const float w = q4.x * qinv, x = q4.y * qinv, y = q4.z * qinv, z = q4.w * qinv;
    const float R[3][3] = {{1.f - 2.f * (y * y + z * z), 2.f * (x * y - w * z), 2.f * (x * z + w * y)},
                           {2.f * (x * y + w * z), 1.f - 2.f * (x * x + z * z), 2.f * (y * z - w * x)},
                           {2.f * (x * z - w * y), 2.f * (y * z + w * x), 1.f - 2.f * (x * x + y * y)}};
    const float s[3] = {expf(ls[0]), expf(ls[1]), expf(ls[2])};
    float M[3][3];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) M[a][b] = R[a][b] * s[b];
    float t[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) t[a] = f.R[3 * a] * X[0] + f.R[3 * a + 1] * X[1] + f.R[3 * a + 2] * X[2] + f.t[a];
    const float rz = 1.f / t[2];
    const float rxu = t[0] * rz, ryu = t[1] * rz;
    const float rx = fminf(f.limx, fmaxf(-f.limx, rxu)), ry = fminf(f.limy, fmaxf(-f.limy, ryu));
    const bool clx = rx != rxu, cly = ry != ryu;
    const float j00 = f.fx * rz, j02 = -f.fx * rx * rz, j11 = f.fy * rz, j12 = -f.fy * ry * rz;
    float Tm[2][3];
#pragma unroll
    for (int b = 0; b < 3; ++b) {
        Tm[0][b] = j00 * f.R[b] + j02 * f.R[6 + b];
        Tm[1][b] = j11 * f.R[3 + b] + j12 * f.R[6 + b];
    }
    // V = Tm M; Sigma' = V V^T + dilation I
    float V[2][3];
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int k = 0; k < 3; ++k) V[a][k] = Tm[a][0] * M[0][k] + Tm[a][1] * M[1][k] + Tm[a][2] * M[2][k];
    const float sxx = V[0][0] * V[0][0] + V[0][1] * V[0][1] + V[0][2] * V[0][2] + f.dilation;
    const float sxy = V[0][0] * V[1][0] + V[0][1] * V[1][1] + V[0][2] * V[1][2];
    const float syy = V[1][0] * V[1][0] + V[1][1] * V[1][1] + V[1][2] * V[1][2] + f.dilation;

    // conic C = Sigma'^{-1} = [[syy, -sxy], [-sxy, sxx]] / D. In the axis
    // basis Ce = [[alpha, beta], [beta, gamma]]: gamma = e2^T C e2 (the large
    // eigenvalue's side), beta = e1^T C e2 (small: the basis is the axes'
    // to rounding), alpha = (det C + beta^2) / gamma with det C = 1 / D, not
    // e1^T C e1, which would cancel.
    const float D = sigma2d_det(V[0], V[1], sxx, syy, f.dilation), iD = 1.f / D;
    const float ca = syy * iD, cb = -sxy * iD, cc = sxx * iD;
    float ct, st;
    axis_basis(axis_t, ct, st);
    const float ce2x = fmaf(cb, ct, -ca * st), ce2y = fmaf(cc, ct, -cb * st);  // C e2
    const float gam = fmaf(ct, ce2y, -st * ce2x);
    const float bet = fmaf(ct, ce2x, st * ce2y);
    const float alp = fmaf(bet, bet, iD) / gam;
    // dL/dSigma_e = -Ce G Ce with G = [[g00, g01], [g01, g11]] = dL/dCe
    const float g00 = pr[2], g01 = 0.5f * pr[3], g11 = pr[4];
    const float m00 = fmaf(g00, alp, g01 * bet), m01 = fmaf(g00, bet, g01 * gam);
    const float m10 = fmaf(g01, alp, g11 * bet), m11 = fmaf(g01, bet, g11 * gam);
    const float h00 = -fmaf(alp, m00, bet * m10), h01 = -fmaf(alp, m01, bet * m11);
    const float h11 = -fmaf(bet, m01, gam * m11);
    // back to x, y: dL/dSigma' = E H E^T with E = [e1 e2] = [[ct, -st], [st, ct]]
    const float cs = ct * st, c2 = ct * ct, s2 = st * st;
    const float G2xy = fmaf(cs, h00 - h11, (c2 - s2) * h01);
    const float G2[2][2] = {{fmaf(c2, h00, fmaf(s2, h11, -2.f * cs * h01)), G2xy},
                            {G2xy, fmaf(s2, h00, fmaf(c2, h11, 2.f * cs * h01))}};
    // Sigma' = V V^T: dV = 2 G2 V; V = Tm M: dTm = dV M^T, dM = Tm^T dV
    float dV[2][3];
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int k = 0; k < 3; ++k) dV[a][k] = 2.f * (G2[a][0] * V[0][k] + G2[a][1] * V[1][k]);
    float GT[2][3];
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) GT[a][b] = dV[a][0] * M[b][0] + dV[a][1] * M[b][1] + dV[a][2] * M[b][2];
    // Tm = J W: dJ = GT W^T (entries 00, 02, 11, 12 are the live ones)
    const float gj00 = GT[0][0] * f.R[0] + GT[0][1] * f.R[1] + GT[0][2] * f.R[2];
    const float gj02 = GT[0][0] * f.R[6] + GT[0][1] * f.R[7] + GT[0][2] * f.R[8];
    const float gj11 = GT[1][0] * f.R[3] + GT[1][1] * f.R[4] + GT[1][2] * f.R[5];
    const float gj12 = GT[1][0] * f.R[6] + GT[1][1] * f.R[7] + GT[1][2] * f.R[8];
    const float rz2 = rz * rz;
    float gt[3] = {0.f, 0.f, 0.f};
    gt[2] += -gj00 * f.fx * rz2 - gj11 * f.fy * rz2;
    if (!clx) { gt[0] += -gj02 * f.fx * rz2; gt[2] += 2.f * gj02 * f.fx * rx * rz2; }
    else gt[2] += gj02 * f.fx * rx * rz2;
    if (!cly) { gt[1] += -gj12 * f.fy * rz2; gt[2] += 2.f * gj12 * f.fy * ry * rz2; }
    else gt[2] += gj12 * f.fy * ry * rz2;
    // projected centre m = (fx tx/tz + cx, fy ty/tz + cy)
    gt[0] += pr[0] * f.fx * rz;
    gt[1] += pr[1] * f.fy * rz;
    gt[2] -= (pr[0] * f.fx * t[0] + pr[1] * f.fy * t[1]) * rz2;
#pragma unroll
    for (int a = 0; a < 3; ++a) gm[a] += f.R[a] * gt[0] + f.R[3 + a] * gt[1] + f.R[6 + a] * gt[2];
    // M = R diag(s): dM = Tm^T dV
    float GR[3][3];
#pragma unroll
    for (int b = 0; b < 3; ++b) {
        float dsb = 0.f;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const float gma = Tm[0][a] * dV[0][b] + Tm[1][a] * dV[1][b];
            dsb = fmaf(gma, R[a][b], dsb);
            GR[a][b] = gma * s[b];
        }
        gls[b] += dsb * s[b];
    }
    float gqh[4];
    gqh[0] = 2.f * (-z * GR[0][1] + y * GR[0][2] + z * GR[1][0] - x * GR[1][2] - y * GR[2][0] + x * GR[2][1]);
    gqh[1] = 2.f * (y * GR[0][1] + z * GR[0][2] + y * GR[1][0] - 2.f * x * GR[1][1] - w * GR[1][2] +
                    z * GR[2][0] + w * GR[2][1] - 2.f * x * GR[2][2]);
    gqh[2] = 2.f * (-2.f * y * GR[0][0] + x * GR[0][1] + w * GR[0][2] + x * GR[1][0] + z * GR[1][2] -
                    w * GR[2][0] + z * GR[2][1] - 2.f * y * GR[2][2]);
    gqh[3] = 2.f * (-2.f * z * GR[0][0] - w * GR[0][1] + x * GR[0][2] + w * GR[1][0] - 2.f * z * GR[1][1] +
                    y * GR[1][2] + x * GR[2][0] + y * GR[2][1]);
    const float qh[4] = {w, x, y, z};
    const float qd = gqh[0] * w + gqh[1] * x + gqh[2] * y + gqh[3] * z;
#pragma unroll
    for (int a = 0; a < 4; ++a) gq[a] += (gqh[a] - qd * qh[a]) * qinv;
}

// Adjoint of the SH colour for one view: pr[6..8] = dL/drgb (zeroed where the
// channel was clamped at 0, detected from the stored colour), `coef` the 48
// coefficients (16-byte aligned). ADDS the direction term into gm and writes
// dL/dcoef into gsh[48] (or adds to it when accumulate is true).
__device__ __forceinline__ void sh_adjoint(const Frame& f, const float X[3], const float* coef, const float rgb[3],
                                           const float pr[9], float gm[3], float* gsh, bool accumulate) {
    const float dx = X[0] - f.campos[0], dy = X[1] - f.campos[1], dz = X[2] - f.campos[2];
    const float invn = rsqrtf(dx * dx + dy * dy + dz * dz);
    const float d[3] = {dx * invn, dy * invn, dz * invn};
    float Y[16], dY[16][3];
    sh_basis_grad(d[0], d[1], d[2], Y, dY);
    float gd[3] = {0.f, 0.f, 0.f};
    float gcol[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) gcol[c] = rgb[c] > 0.f ? pr[6 + c] : 0.f;
#pragma unroll
    for (int k = 0; k < 16; ++k) {
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const float cf = coef[3 * k + c];
            gd[0] = fmaf(cf * gcol[c], dY[k][0], gd[0]);
            gd[1] = fmaf(cf * gcol[c], dY[k][1], gd[1]);
            gd[2] = fmaf(cf * gcol[c], dY[k][2], gd[2]);
        }
    }
#pragma unroll
    for (int k = 0; k < 16; ++k)
#pragma unroll
        for (int c = 0; c < 3; ++c) gsh[3 * k + c] = accumulate ? gsh[3 * k + c] + Y[k] * gcol[c] : Y[k] * gcol[c];
    const float dd = gd[0] * d[0] + gd[1] * d[1] + gd[2] * d[2];
#pragma unroll
    for (int a = 0; a < 3; ++a) gm[a] += (gd[a] - dd * d[a]) * invn;
}

}  // namespace ws
