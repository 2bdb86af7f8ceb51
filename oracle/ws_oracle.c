/*
 * FP64 CPU oracle for the per-frame 3D Gaussian Splatting render path of
 * "WebSplatter: Enabling Cross-Device Efficient Gaussian Splatting in Web
 * Browsers via WebGPU" (arXiv 2602.03207).
 *
 * TEST INFRASTRUCTURE. Only the tests, the smoke check and the benchmark's
 * CPU-baseline leg load this code; the library never does. It shares no code,
 * header, table or constant generator with the CUDA path. It is written to be
 * read against the paper, not to be fast: plain loops, double precision, no
 * blocking or fusion beyond what the paper's definitions state.
 *
 * What it computes, and where the paper defines it:
 *   or_sh_basis         SH colour basis, §2.1 (c_i = SH(k_i, d)), real SH
 *                       written from the associated-Legendre definition.
 *   or_sh_basis_cart    the same 16 functions as Cartesian polynomials with
 *                       their gradient (used by the backward; pinned against
 *                       or_sh_basis in the tests).
 *   or_preprocess       §2.1 density/covariance and splat alpha, §3.2
 *                       projection + AABB culling + 32-bit float depth,
 *                       §3.4 opacity culling (sigma < 1/255) and the
 *                       opacity-aware extent (1/255 = sigma e^{-r^2}).
 *                       With OR_PACKED, the record is packed first (§3.2):
 *                       opacity and clamped colour on 8 bits, the centre in
 *                       float32, the ellipse as two binary16 axes
 *                       (or_round_f16, or_axes), and Sigma', the conic and
 *                       the extent follow from the packed values.
 *   or_emit_keys        the <tile, splat> pair list of §3.4 (the CUDA-style
 *                       tile decomposition), one key per overlapped tile.
 *   or_sort_pairs       §3.3.2: a stable sort (elements with equal keys keep
 *                       their input order). Bottom-up merge sort.
 *   or_tile_ranges      [start, end) of every tile in the sorted pair list.
 *   or_blend_tiles      §2.1 compositing C = sum c_i a_i prod_{j<i}(1 - a_j),
 *                       front to back over each tile's depth-sorted list.
 *   or_blend_brute      the same per pixel over ALL visible splats, back to
 *                       front with the "over" operator (§2.1 states the
 *                       back-to-front order; §3.3 hardware blending).
 *   or_loss_grad        L = 1/2 ||C - target||^2 and its analytic FP64
 *                       gradient w.r.t. every input (the paper renders only;
 *                       §1 notes 3DGS is differentiable).
 *
 * Readings where the paper is silent:
 *   - parameterisation: s = exp(log_scale), q = (w,x,y,z) normalised,
 *     sigma = 1 / (1 + exp(-logit)); Sigma = R diag(s^2) R^T.
 *   - projection: pinhole with OpenCV axes, pixel u spans [u, u+1) and its
 *     centre is u + 1/2; EWA local affine Jacobian J of the perspective map
 *     with t_x/t_z, t_y/t_z clamped to +-guard*(W/2)/f_x, +-guard*(H/2)/f_y
 *     inside J only; Sigma' = J W Sigma W^T J^T + dilation * I.
 *   - the splat alpha of §2.1 is a = min(0.99, sigma exp(-q/2)),
 *     q = x'^T Sigma'^{-1} x'; a pair with a < 1/255 is skipped (the paper's
 *     quantisation threshold). The cutoff equation of §3.4 writes e^{-r^2}:
 *     read as r^2 = q/2, so the extent where a = 1/255 is q_c = 2 ln(255 sigma).
 *   - opacity cull: sigma < 1/255 (strict, per §3.4), decided as
 *     logit < -ln(254) on the float32 input.
 *   - depth: the float32 value t_z = ((r20*x + r21*y) + r22*z) + t2
 *     evaluated in float32 with each operation rounded (§3.2 stores depth as a
 *     32-bit float). The near plane test and the sort key use this value.
 *   - order of equal depths: ascending Gaussian index (the stable sort).
 *   - SH: real SH with the Condon-Shortley phase, index l^2 + l + m; colour
 *     c = max(0, sum_lm k_lm Y_lm(d) + 1/2), d = normalise(X - camera centre).
 *   - sort key: (tile id << 31) | float32 bits of the depth (sign bit 0).
 *
 * Ambiguity: decisions taken on floating-point values (tile bounds, the
 * viewport test, the per-pixel 1/255 test) can fall either way within the
 * float32 error of the GPU. The oracle reports, per decision, whether it lies
 * within a relative margin of its threshold; tests then demand exact
 * agreement on every unambiguous decision and accept either outcome of an
 * ambiguous one (the alternative image is computed for pixels with one).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

typedef struct {
    double viewmat[12]; /* row-major 3x4 [R | t], world -> camera */
    double fx, fy, cx, cy;
    int32_t width, height;
    double znear;
    double bg[3];
} or_camera;

typedef struct {
    int32_t tile;        /* tile side in pixels */
    double dilation;     /* px^2 added to the diagonal of Sigma' */
    double guard;        /* frustum guard factor of the Jacobian clamp */
    double amb_px_rel;   /* relative margin of tile-bound / viewport decisions */
    double amb_alpha;    /* relative margin of the per-pixel 1/255 decision */
    int32_t flags;       /* ablations (§4.4): 1 keep sigma < 1/255, 2 keep off-screen boxes, 8 fixed extent;
                            16 packed record (§3.2) */
} or_config;

enum { OR_NO_OPACITY_CULL = 1, OR_NO_AABB_CULL = 2, OR_FIXED_RADIUS = 8, OR_PACKED = 16 };

enum { OR_VISIBLE = 0, OR_CULL_OPACITY = 1, OR_CULL_QUAT = 2, OR_CULL_NEAR = 3,
       OR_CULL_DET = 4, OR_CULL_OFFSCREEN = 5 };

/* ---------------------------------------------------------------- helpers */

static double fact(int k) { double r = 1.0; for (int i = 2; i <= k; ++i) r *= i; return r; }

static int tiles_x(const or_camera *c, const or_config *g) { return (c->width + g->tile - 1) / g->tile; }
static int tiles_y(const or_camera *c, const or_config *g) { return (c->height + g->tile - 1) / g->tile; }

/* Real-valued SH basis of degree <= 3 from its definition (§2.1 colour):
 *   Y_l^m = (-1)^m sqrt(2) K_l^|m| P_l^|m|(cos th) cos(m phi)      m > 0
 *   Y_l^0 = K_l^0 P_l^0(cos th)
 *   Y_l^m = (-1)^m sqrt(2) K_l^|m| P_l^|m|(cos th) sin(|m| phi)    m < 0
 * with K_l^m = sqrt((2l+1)/(4 pi) (l-m)!/(l+m)!) and P_l^m the associated
 * Legendre function without the Condon-Shortley phase (which is the
 * (-1)^m factor above). Output index l*l + l + m. d must be unit length. */
void or_sh_basis(const double d[3], double Y[16])
{
    double z = d[2];
    double st = sqrt(fmax(0.0, 1.0 - z * z));
    double phi = atan2(d[1], d[0]);
    double P[4][4] = {{0}};
    for (int m = 0; m <= 3; ++m) {
        double pmm = 1.0;
        for (int k = 1; k <= m; ++k) pmm *= (2.0 * k - 1.0) * st; /* (2m-1)!! sin^m */
        P[m][m] = pmm;
        if (m + 1 <= 3) P[m + 1][m] = z * (2.0 * m + 1.0) * pmm;
        for (int l = m + 2; l <= 3; ++l)
            P[l][m] = ((2.0 * l - 1.0) * z * P[l - 1][m] - (l + m - 1.0) * P[l - 2][m]) / (l - m);
    }
    for (int l = 0; l <= 3; ++l) {
        for (int m = -l; m <= l; ++m) {
            int am = m < 0 ? -m : m;
            double K = sqrt((2.0 * l + 1.0) / (4.0 * M_PI) * fact(l - am) / fact(l + am));
            double v;
            if (m == 0) v = K * P[l][0];
            else if (m > 0) v = sqrt(2.0) * K * cos(m * phi) * P[l][am];
            else v = sqrt(2.0) * K * sin(am * phi) * P[l][am];
            if (am & 1) v = -v;
            Y[l * l + l + m] = v;
        }
    }
}

/* The same 16 functions written as homogeneous Cartesian polynomials in
 * (x, y, z), with the gradient of each polynomial. Used by the backward
 * (the direction gradient). Values agree with or_sh_basis on the unit
 * sphere; the tests pin that. Constants are the K factors above, evaluated. */
void or_sh_basis_cart(const double d[3], double Y[16], double dY[16][3])
{
    double x = d[0], y = d[1], z = d[2];
    double k0 = sqrt(1.0 / (4.0 * M_PI));
    double k1 = sqrt(3.0 / (4.0 * M_PI));
    double k2a = sqrt(15.0 / (4.0 * M_PI));   /* xy, yz, xz */
    double k2b = sqrt(5.0 / (16.0 * M_PI));   /* 2z^2 - x^2 - y^2 */
    double k2c = sqrt(15.0 / (16.0 * M_PI));  /* x^2 - y^2 */
    double k3a = sqrt(35.0 / (32.0 * M_PI));  /* y(3x^2 - y^2), x(x^2 - 3y^2) */
    double k3b = sqrt(105.0 / (4.0 * M_PI));  /* xyz */
    double k3c = sqrt(21.0 / (32.0 * M_PI));  /* y(4z^2 - x^2 - y^2), x(...) */
    double k3d = sqrt(7.0 / (16.0 * M_PI));   /* z(2z^2 - 3x^2 - 3y^2) */
    double k3e = sqrt(105.0 / (16.0 * M_PI)); /* z(x^2 - y^2) */
    double v[16], g[16][3];
    memset(g, 0, sizeof(g));
    v[0] = k0;
    v[1] = -k1 * y;  g[1][1] = -k1;
    v[2] = k1 * z;   g[2][2] = k1;
    v[3] = -k1 * x;  g[3][0] = -k1;
    v[4] = k2a * x * y;            g[4][0] = k2a * y; g[4][1] = k2a * x;
    v[5] = -k2a * y * z;           g[5][1] = -k2a * z; g[5][2] = -k2a * y;
    v[6] = k2b * (2 * z * z - x * x - y * y);
    g[6][0] = -2 * k2b * x; g[6][1] = -2 * k2b * y; g[6][2] = 4 * k2b * z;
    v[7] = -k2a * x * z;           g[7][0] = -k2a * z; g[7][2] = -k2a * x;
    v[8] = k2c * (x * x - y * y);  g[8][0] = 2 * k2c * x; g[8][1] = -2 * k2c * y;
    v[9] = -k3a * y * (3 * x * x - y * y);
    g[9][0] = -k3a * 6 * x * y; g[9][1] = -k3a * (3 * x * x - 3 * y * y);
    v[10] = k3b * x * y * z;
    g[10][0] = k3b * y * z; g[10][1] = k3b * x * z; g[10][2] = k3b * x * y;
    v[11] = -k3c * y * (4 * z * z - x * x - y * y);
    g[11][0] = k3c * 2 * x * y; g[11][1] = -k3c * (4 * z * z - x * x - 3 * y * y);
    g[11][2] = -k3c * 8 * y * z;
    v[12] = k3d * z * (2 * z * z - 3 * x * x - 3 * y * y);
    g[12][0] = -k3d * 6 * x * z; g[12][1] = -k3d * 6 * y * z;
    g[12][2] = k3d * (6 * z * z - 3 * x * x - 3 * y * y);
    v[13] = -k3c * x * (4 * z * z - x * x - y * y);
    g[13][0] = -k3c * (4 * z * z - 3 * x * x - y * y); g[13][1] = k3c * 2 * x * y;
    g[13][2] = -k3c * 8 * x * z;
    v[14] = k3e * z * (x * x - y * y);
    g[14][0] = k3e * 2 * x * z; g[14][1] = -k3e * 2 * y * z; g[14][2] = k3e * (x * x - y * y);
    v[15] = -k3a * x * (x * x - 3 * y * y);
    g[15][0] = -k3a * (3 * x * x - 3 * y * y); g[15][1] = k3a * 6 * x * y;
    for (int i = 0; i < 16; ++i) {
        Y[i] = v[i];
        if (dY) { dY[i][0] = g[i][0]; dY[i][1] = g[i][1]; dY[i][2] = g[i][2]; }
    }
}

/* Rotation matrix of a unit quaternion (w, x, y, z) (§2.1: Sigma is built
 * from a rotation quaternion and a scaling vector). */
static void quat_to_rot(const double q[4], double R[3][3])
{
    double w = q[0], x = q[1], y = q[2], z = q[3];
    R[0][0] = 1 - 2 * (y * y + z * z); R[0][1] = 2 * (x * y - w * z); R[0][2] = 2 * (x * z + w * y);
    R[1][0] = 2 * (x * y + w * z); R[1][1] = 1 - 2 * (x * x + z * z); R[1][2] = 2 * (y * z - w * x);
    R[2][0] = 2 * (x * z - w * y); R[2][1] = 2 * (y * z + w * x); R[2][2] = 1 - 2 * (x * x + y * y);
}

/* The float32 view depth of §3.2, evaluated in float32 with every operation
 * rounded in the stated order (no fused multiply-add). */
float or_depth32(const double X[3], const double viewmat[12])
{
    volatile float a = (float)viewmat[8] * (float)X[0];
    volatile float b = (float)viewmat[9] * (float)X[1];
    volatile float s = a + b;
    volatile float c = (float)viewmat[10] * (float)X[2];
    volatile float s2 = s + c;
    volatile float r = s2 + (float)viewmat[11];
    return r;
}

static double tau_opacity(void) { return -log(254.0); } /* sigma < 1/255 <=> logit < -ln 254 */

/* ----------------------------------------------------------- packed record
 * §3.2 packs a splat's colour and opacity into one RGBA8 word and its
 * ellipse axes into two words of two IEEE binary16 halves each. */

/* Round to the nearest binary16 value, ties to even, from double directly
 * (no intermediate float). Overflow gives +-inf. */
double or_round_f16(double x)
{
    if (x == 0.0 || isnan(x) || isinf(x)) return x;
    double ax = fabs(x);
    int e;
    frexp(ax, &e);                      /* ax = f 2^e, f in [0.5, 1) */
    int ulp_exp = e - 11;               /* 11 significant bits */
    if (ulp_exp < -24) ulp_exp = -24;   /* subnormal halves: spacing 2^-24 */
    double q = ldexp(rint(ldexp(ax, -ulp_exp)), ulp_exp);
    if (q >= 65520.0) q = INFINITY;     /* 65520 rounds up past the largest half, 65504 */
    return x < 0 ? -q : q;
}

/* x in [0, 1] on 8 bits: the nearest multiple of 1/255, ties to even. */
static double quant8(double x)
{
    if (x < 0.0) x = 0.0;
    if (x > 1.0) x = 1.0;
    return rint(x * 255.0) / 255.0;
}

/* Ellipse axes of the 2D covariance [[sxx, sxy], [sxy, syy]]: v1 = sqrt(l1) e1
 * (major), v2 = sqrt(l2) e2 (minor, e2 = e1 turned by +90 degrees), so that
 * Sigma' = v1 v1^T + v2 v2^T. e1 comes from whichever row of (Sigma' - l1 I)
 * is better conditioned; l2 = det / l1 avoids the cancellation of m - d. */
void or_axes(double sxx, double sxy, double syy, double *v1, double *v2)
{
    double m = 0.5 * (sxx + syy), h = 0.5 * (sxx - syy);
    double d = sqrt(h * h + sxy * sxy);
    double l1 = m + d, l2 = (sxx * syy - sxy * sxy) / l1;
    double ex = 1.0, ey = 0.0;
    if (d > 0.0) {
        if (h >= 0.0) { double nn = hypot(d + h, sxy); ex = (d + h) / nn; ey = sxy / nn; }
        else { double nn = hypot(sxy, d - h); ex = sxy / nn; ey = (d - h) / nn; }
    }
    double r1 = sqrt(l1), r2 = sqrt(l2);
    v1[0] = r1 * ex; v1[1] = r1 * ey;
    v2[0] = -r2 * ey; v2[1] = r2 * ex;
}

static double flr(double v) { return floor(v); }

/* ------------------------------------------------------------ preprocess */

/* Per-Gaussian pre-processing (§3.2 with §2.1 and §3.4):
 * activation, projection of the centre and covariance to the image, SH
 * colour, opacity cull, near-plane cull, opacity-aware extent, viewport
 * AABB cull and the tile rectangle it overlaps.
 *
 * Outputs (all per Gaussian):
 *   mean2d[2], cov2d[3] (Sigma' xx, xy, yy incl. dilation), conic[3]
 *   (Sigma'^{-1} a, b, c), depth32, rgb[3], opacity (sigma), extent[2],
 *   rect[4] = tile x0, y0, x1, y1 inclusive (canonical decisions; empty
 *   (x0 > x1) when culled), rect_exp[4] = rect widened by the ambiguity
 *   margin (also set for a splat whose off-screen cull is ambiguous),
 *   touched = tiles in rect, reason (OR_*), amb = 1 if any tile-bound or
 *   viewport decision lies within the margin.
 * Returns the number of visible Gaussians. */
int64_t or_preprocess(int64_t n, const double *means, const double *log_scales,
                      const double *quats, const double *logits, const double *sh,
                      const or_camera *cam, const or_config *cfg,
                      double *mean2d, double *cov2d, double *conic, float *depth32,
                      double *rgb, double *opacity, double *extent,
                      int32_t *rect, int32_t *rect_exp, int32_t *touched,
                      int32_t *reason, uint8_t *amb)
{
    const double *V = cam->viewmat;
    double Rv[3][3] = {{V[0], V[1], V[2]}, {V[4], V[5], V[6]}, {V[8], V[9], V[10]}};
    double tv[3] = {V[3], V[7], V[11]};
    double campos[3];
    for (int i = 0; i < 3; ++i)
        campos[i] = -(Rv[0][i] * tv[0] + Rv[1][i] * tv[1] + Rv[2][i] * tv[2]);
    const int TS = cfg->tile, TX = tiles_x(cam, cfg), TY = tiles_y(cam, cfg);
    const double W = cam->width, H = cam->height;
    const double limx = cfg->guard * 0.5 * W / cam->fx, limy = cfg->guard * 0.5 * H / cam->fy;
    int64_t visible = 0;

    for (int64_t i = 0; i < n; ++i) {
        int32_t *rc = rect + 4 * i, *re = rect_exp + 4 * i;
        rc[0] = re[0] = 0; rc[1] = re[1] = 0; rc[2] = re[2] = -1; rc[3] = re[3] = -1;
        touched[i] = 0; amb[i] = 0;
        const double *X = means + 3 * i;
        depth32[i] = or_depth32(X, V);
        double logit = logits[i];
        double sigma = 1.0 / (1.0 + exp(-logit));
        opacity[i] = sigma;
        if (logit < tau_opacity() && !(cfg->flags & OR_NO_OPACITY_CULL)) { reason[i] = OR_CULL_OPACITY; continue; }
        const double *q0 = quats + 4 * i;
        double qn = sqrt(q0[0] * q0[0] + q0[1] * q0[1] + q0[2] * q0[2] + q0[3] * q0[3]);
        if (qn == 0.0) { reason[i] = OR_CULL_QUAT; continue; }
        if (depth32[i] <= (float)cam->znear) { reason[i] = OR_CULL_NEAR; continue; }

        /* 3D covariance Sigma = R S S^T R^T (§2.1). */
        double q[4] = {q0[0] / qn, q0[1] / qn, q0[2] / qn, q0[3] / qn};
        double R[3][3];
        quat_to_rot(q, R);
        double s[3] = {exp(log_scales[3 * i]), exp(log_scales[3 * i + 1]), exp(log_scales[3 * i + 2])};
        double Sig[3][3];
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) {
                double acc = 0;
                for (int k = 0; k < 3; ++k) acc += R[a][k] * s[k] * s[k] * R[b][k];
                Sig[a][b] = acc;
            }
        /* Camera-space centre t = W X + t_v and projected centre (§3.2). */
        double t[3];
        for (int a = 0; a < 3; ++a) t[a] = Rv[a][0] * X[0] + Rv[a][1] * X[1] + Rv[a][2] * X[2] + tv[a];
        double mx = cam->fx * t[0] / t[2] + cam->cx;
        double my = cam->fy * t[1] / t[2] + cam->cy;
        /* EWA Jacobian with the guard-band clamp. */
        double rx = t[0] / t[2], ry = t[1] / t[2];
        if (rx < -limx) rx = -limx;
        if (rx > limx) rx = limx;
        if (ry < -limy) ry = -limy;
        if (ry > limy) ry = limy;
        double J[2][3] = {{cam->fx / t[2], 0.0, -cam->fx * rx / t[2]},
                          {0.0, cam->fy / t[2], -cam->fy * ry / t[2]}};
        double T[2][3];
        for (int a = 0; a < 2; ++a)
            for (int b = 0; b < 3; ++b)
                T[a][b] = J[a][0] * Rv[0][b] + J[a][1] * Rv[1][b] + J[a][2] * Rv[2][b];
        double C2[2][2];
        for (int a = 0; a < 2; ++a)
            for (int b = 0; b < 2; ++b) {
                double acc = 0;
                for (int k = 0; k < 3; ++k)
                    for (int l = 0; l < 3; ++l) acc += T[a][k] * Sig[k][l] * T[b][l];
                C2[a][b] = acc;
            }
        double sxx = C2[0][0] + cfg->dilation, sxy = C2[0][1], syy = C2[1][1] + cfg->dilation;
        double det = sxx * syy - sxy * sxy;
        mean2d[2 * i] = mx; mean2d[2 * i + 1] = my;
        cov2d[3 * i] = sxx; cov2d[3 * i + 1] = sxy; cov2d[3 * i + 2] = syy;
        if (!(det > 0.0)) { reason[i] = OR_CULL_DET; continue; }
        conic[3 * i] = syy / det; conic[3 * i + 1] = -sxy / det; conic[3 * i + 2] = sxx / det;

        /* SH colour along the camera-to-centre direction (§2.1, §3.2). */
        double dir[3] = {X[0] - campos[0], X[1] - campos[1], X[2] - campos[2]};
        double dn = sqrt(dir[0] * dir[0] + dir[1] * dir[1] + dir[2] * dir[2]);
        dir[0] /= dn; dir[1] /= dn; dir[2] /= dn;
        double Y[16];
        or_sh_basis(dir, Y);
        for (int ch = 0; ch < 3; ++ch) {
            double acc = 0.0;
            for (int k = 0; k < 16; ++k) acc += Y[k] * sh[(16 * i + k) * 3 + ch];
            acc += 0.5;
            rgb[3 * i + ch] = acc > 0.0 ? acc : 0.0;
        }

        if (cfg->flags & OR_PACKED) {
            /* Packed record (§3.2): opacity and clamped colour on 8 bits, the
             * centre in float32, the ellipse as two binary16 axes; Sigma',
             * the conic and the extent below follow from the packed values. */
            sigma = quant8(sigma);
            opacity[i] = sigma;
            for (int ch = 0; ch < 3; ++ch) rgb[3 * i + ch] = quant8(rgb[3 * i + ch]);
            mx = (double)(float)mx; my = (double)(float)my;
            mean2d[2 * i] = mx; mean2d[2 * i + 1] = my;
            double v1[2], v2[2];
            or_axes(sxx, sxy, syy, v1, v2);
            for (int a = 0; a < 2; ++a) { v1[a] = or_round_f16(v1[a]); v2[a] = or_round_f16(v2[a]); }
            sxx = v1[0] * v1[0] + v2[0] * v2[0];
            sxy = v1[0] * v1[1] + v2[0] * v2[1];
            syy = v1[1] * v1[1] + v2[1] * v2[1];
            double cross = v1[0] * v2[1] - v1[1] * v2[0];
            det = cross * cross;
            cov2d[3 * i] = sxx; cov2d[3 * i + 1] = sxy; cov2d[3 * i + 2] = syy;
            if (!(det > 0.0)) { reason[i] = OR_CULL_DET; continue; }
            conic[3 * i] = syy / det; conic[3 * i + 1] = -sxy / det; conic[3 * i + 2] = sxx / det;
        }

        /* Opacity-aware extent (§3.4): a >= 1/255 <=> q <= q_c = 2 ln(255 sigma).
         * The axis-aligned box of the ellipse x^T Sigma'^{-1} x <= q_c has
         * half-widths sqrt(q_c Sigma'_xx), sqrt(q_c Sigma'_yy). */
        double qc = 2.0 * log(255.0 * sigma);
        if (qc < 0.0) qc = 0.0;
        /* ablation "-RADIUS" (§4.4, Table 5): a box independent of the
         * opacity, the one a splat of sigma = 1 needs */
        if (cfg->flags & OR_FIXED_RADIUS) qc = 2.0 * log(255.0);
        double ex = sqrt(qc * sxx), ey = sqrt(qc * syy);
        extent[2 * i] = ex; extent[2 * i + 1] = ey;

        double eps = cfg->amb_px_rel * (fabs(mx) + fabs(my) + ex + ey + TS);
        double lo[2] = {mx - ex, my - ey}, hi[2] = {mx + ex, my + ey};
        double lim[2] = {W, H};
        /* Viewport AABB test (§3.2): [m - e, m + e] must meet [0, W) x [0, H). */
        int on = 1, on_relaxed = 1;
        for (int a = 0; a < 2; ++a) {
            if (!(hi[a] >= 0.0 && lo[a] < lim[a])) on = 0;
            if (!(hi[a] >= -eps && lo[a] < lim[a] + eps)) on_relaxed = 0;
            if (fabs(hi[a]) < eps || fabs(lo[a] - lim[a]) < eps) amb[i] = 1;
        }
        if (on_relaxed || (cfg->flags & OR_NO_AABB_CULL)) {
            /* Widened rectangle: every tile either rounding could select. */
            int x0 = (int)fmin(TX - 1.0, fmax(0.0, flr((lo[0] - eps) / TS)));
            int x1 = (int)fmin(TX - 1.0, fmax(0.0, flr((hi[0] + eps) / TS)));
            int y0 = (int)fmin(TY - 1.0, fmax(0.0, flr((lo[1] - eps) / TS)));
            int y1 = (int)fmin(TY - 1.0, fmax(0.0, flr((hi[1] + eps) / TS)));
            re[0] = x0; re[1] = y0; re[2] = x1; re[3] = y1;
        }
        /* ablation "-CULL" (§4.4): off-screen boxes are kept, clamped to the screen */
        if (!on && !(cfg->flags & OR_NO_AABB_CULL)) { reason[i] = OR_CULL_OFFSCREEN; continue; }
        /* Tile rectangle: tiles whose column / row range holds a pixel centre
         * of [m - e, m + e] (tile k covers [k TS, (k+1) TS)). */
        int x0 = (int)fmin(TX - 1.0, fmax(0.0, flr(lo[0] / TS))), x1 = (int)fmin(TX - 1.0, fmax(0.0, flr(hi[0] / TS)));
        int y0 = (int)fmin(TY - 1.0, fmax(0.0, flr(lo[1] / TS))), y1 = (int)fmin(TY - 1.0, fmax(0.0, flr(hi[1] / TS)));
        for (int a = 0; a < 2; ++a) {
            double vv[2] = {lo[a], hi[a]};
            int ntile = a == 0 ? TX : TY;
            for (int k = 0; k < 2; ++k) {
                /* nearest tile boundary; the outer ones are clamped either way */
                double b = TS * flr(vv[k] / TS + 0.5);
                if (b <= 0.0 || b >= (double)ntile * TS) continue;
                if (fabs(vv[k] - b) < eps) amb[i] = 1;
            }
        }
        rc[0] = x0; rc[1] = y0; rc[2] = x1; rc[3] = y1;
        touched[i] = (x1 - x0 + 1) * (y1 - y0 + 1);
        reason[i] = OR_VISIBLE;
        ++visible;
    }
    return visible;
}

/* ------------------------------------------------------------ key emission */

/* The <tile, splat> pair list (§3.4; the tile decomposition): for every
 * Gaussian i in index order with a non-empty rect, and every tile of the
 * rect in row-major order, key = (tile id << 31) | bits(depth32_i), val = i.
 * offsets[i] = first slot of Gaussian i (exclusive scan of the tile counts);
 * offsets has n + 1 entries. Returns the number of keys. */
int64_t or_emit_keys(int64_t n, const int32_t *rect, const float *depth32, int32_t tiles_x_,
                     uint64_t *keys, uint32_t *vals, int64_t *offsets)
{
    int64_t k = 0;
    for (int64_t i = 0; i < n; ++i) {
        if (offsets) offsets[i] = k;
        const int32_t *r = rect + 4 * i;
        if (r[0] > r[2] || r[1] > r[3]) continue;
        uint32_t bits;
        memcpy(&bits, &depth32[i], 4);
        for (int ty = r[1]; ty <= r[3]; ++ty)
            for (int tx = r[0]; tx <= r[2]; ++tx) {
                uint64_t tile = (uint64_t)ty * (uint64_t)tiles_x_ + (uint64_t)tx;
                if (keys) { keys[k] = (tile << 31) | (uint64_t)(bits & 0x7fffffffu); vals[k] = (uint32_t)i; }
                ++k;
            }
    }
    if (offsets) offsets[n] = k;
    return k;
}

/* ------------------------------------------------------------------ sort */

/* Stable sort of (key, val) pairs by key (§3.3.2: elements with equal keys
 * keep their input order). Plain bottom-up merge sort; the left run wins
 * ties, which is what makes it stable. */
void or_sort_pairs(int64_t n, uint64_t *keys, uint32_t *vals)
{
    if (n < 2) return;
    uint64_t *k2 = (uint64_t *)malloc((size_t)n * sizeof(uint64_t));
    uint32_t *v2 = (uint32_t *)malloc((size_t)n * sizeof(uint32_t));
    uint64_t *ka = keys, *kb = k2;
    uint32_t *va = vals, *vb = v2;
    for (int64_t width = 1; width < n; width *= 2) {
        for (int64_t lo = 0; lo < n; lo += 2 * width) {
            int64_t mid = lo + width < n ? lo + width : n;
            int64_t hi = lo + 2 * width < n ? lo + 2 * width : n;
            int64_t i = lo, j = mid, o = lo;
            while (i < mid && j < hi) {
                if (ka[j] < ka[i]) { kb[o] = ka[j]; vb[o++] = va[j++]; }
                else { kb[o] = ka[i]; vb[o++] = va[i++]; }
            }
            while (i < mid) { kb[o] = ka[i]; vb[o++] = va[i++]; }
            while (j < hi) { kb[o] = ka[j]; vb[o++] = va[j++]; }
        }
        uint64_t *tk = ka; ka = kb; kb = tk;
        uint32_t *tvv = va; va = vb; vb = tvv;
    }
    if (ka != keys) { memcpy(keys, ka, (size_t)n * 8); memcpy(vals, va, (size_t)n * 4); }
    free(k2); free(v2);
}

/* [start, end) of every tile id in a key list sorted by key. */
void or_tile_ranges(int64_t nkeys, const uint64_t *keys, int64_t ntiles, int64_t *ranges)
{
    for (int64_t t = 0; t < ntiles; ++t) { ranges[2 * t] = 0; ranges[2 * t + 1] = 0; }
    for (int64_t p = 0; p < nkeys; ++p) {
        int64_t t = (int64_t)(keys[p] >> 31);
        if (p == 0 || (int64_t)(keys[p - 1] >> 31) != t) ranges[2 * t] = p;
        if (p == nkeys - 1 || (int64_t)(keys[p + 1] >> 31) != t) ranges[2 * t + 1] = p + 1;
    }
}

/* ----------------------------------------------------------------- blend */

/* Splat alpha of §2.1 at pixel centre p for Gaussian g:
 * a = min(0.99, sigma exp(-q/2)), q = d^T Sigma'^{-1} d, d = p - mean2d. */
static double splat_alpha(const double *mean2d, const double *conic, const double *opacity,
                          int64_t g, double px, double py, double *G_out, double *dx_out, double *dy_out)
{
    double dx = px - mean2d[2 * g], dy = py - mean2d[2 * g + 1];
    const double *Q = conic + 3 * g;
    double q = Q[0] * dx * dx + 2.0 * Q[1] * dx * dy + Q[2] * dy * dy;
    double G = exp(-0.5 * q);
    double a = opacity[g] * G;
    if (G_out) *G_out = G;
    if (dx_out) { *dx_out = dx; *dy_out = dy; }
    return a < 0.99 ? a : 0.99;
}

/* Decision of the 1/255 test: 1 include, 0 skip; *ambig = 1 when the value
 * is within the relative margin of the threshold. */
static int alpha_keep(double a, double rel, int *ambig)
{
    const double thr = 1.0 / 255.0;
    *ambig = fabs(a - thr) < rel * thr;
    return a >= thr;
}

/* Front-to-back compositing of §2.1 (C = sum c_i a_i T_i, T_i = prod_{j<i}
 * (1 - a_j)) for every pixel of the listed tiles, each over its tile's
 * depth-sorted list (vals[ranges[t][0] .. ranges[t][1]) ).
 * tile_list == NULL renders all tiles. Per pixel: image[3] = C + T bg,
 * t_final = T, last_gid = index of the last Gaussian composited (-1: none),
 * n_amb = number of ambiguous 1/255 decisions; when n_amb == 1, alt_* hold
 * the result with that single decision flipped. */
void or_blend_tiles(const or_camera *cam, const or_config *cfg,
                    const double *mean2d, const double *conic, const double *opacity,
                    const double *rgb, const uint32_t *vals, const int64_t *ranges,
                    int64_t n_tiles_listed, const int64_t *tile_list,
                    double *image, double *t_final, int64_t *last_gid, int32_t *n_amb,
                    double *alt_image, double *alt_t_final, int64_t *alt_last_gid)
{
    const int TS = cfg->tile, TX = tiles_x(cam, cfg), TY = tiles_y(cam, cfg);
    int64_t ntiles = tile_list ? n_tiles_listed : (int64_t)TX * TY;
    for (int64_t it = 0; it < ntiles; ++it) {
        int64_t t = tile_list ? tile_list[it] : it;
        int tx = (int)(t % TX), ty = (int)(t / TX);
        for (int v = ty * TS; v < (ty + 1) * TS && v < cam->height; ++v)
            for (int u = tx * TS; u < (tx + 1) * TS && u < cam->width; ++u) {
                double px = u + 0.5, py = v + 0.5;
                int64_t pix = (int64_t)v * cam->width + u;
                int64_t flip_at = -1;
                for (int pass = 0; pass < 2; ++pass) {
                    double C[3] = {0, 0, 0}, T = 1.0;
                    int64_t last = -1;
                    int32_t amb_count = 0;
                    for (int64_t j = ranges[2 * t]; j < ranges[2 * t + 1]; ++j) {
                        int64_t g = vals[j];
                        double a = splat_alpha(mean2d, conic, opacity, g, px, py, NULL, NULL, NULL);
                        int ambig;
                        int keep = alpha_keep(a, cfg->amb_alpha, &ambig);
                        if (ambig) { if (pass == 0 && amb_count == 0) flip_at = j; ++amb_count; }
                        if (pass == 1 && j == flip_at) keep = !keep;
                        if (!keep) continue;
                        for (int ch = 0; ch < 3; ++ch) C[ch] += rgb[3 * g + ch] * a * T;
                        T *= 1.0 - a;
                        last = g;
                    }
                    double *img = pass == 0 ? image : alt_image;
                    for (int ch = 0; ch < 3; ++ch) img[3 * pix + ch] = C[ch] + T * cam->bg[ch];
                    if (pass == 0) { t_final[pix] = T; last_gid[pix] = last; n_amb[pix] = amb_count; }
                    else { alt_t_final[pix] = T; alt_last_gid[pix] = last; }
                    if (pass == 0 && amb_count != 1) {
                        for (int ch = 0; ch < 3; ++ch) alt_image[3 * pix + ch] = img[3 * pix + ch];
                        alt_t_final[pix] = T; alt_last_gid[pix] = last;
                        break;
                    }
                }
            }
    }
}

/* Brute force over every visible Gaussian (no tiles): per pixel, sort all
 * splats with touched > 0 by (depth32, index) and composite back to front
 * with the "over" operator, C <- a c + (1 - a) C, starting from the
 * background (§2.1 states the back-to-front order). Same 1/255 rule. */
void or_blend_brute(const or_camera *cam, int64_t n, const double *mean2d, const double *conic,
                    const double *opacity, const double *rgb, const float *depth32,
                    const int32_t *touched, double *image, double *t_final)
{
    int64_t nv = 0;
    uint64_t *k = (uint64_t *)malloc((size_t)(n > 0 ? n : 1) * 8);
    uint32_t *id = (uint32_t *)malloc((size_t)(n > 0 ? n : 1) * 4);
    for (int64_t i = 0; i < n; ++i)
        if (touched[i] > 0) {
            uint32_t bits; memcpy(&bits, &depth32[i], 4);
            k[nv] = bits; id[nv] = (uint32_t)i; ++nv;
        }
    or_sort_pairs(nv, k, id);
    for (int v = 0; v < cam->height; ++v)
        for (int u = 0; u < cam->width; ++u) {
            double px = u + 0.5, py = v + 0.5;
            double C[3] = {cam->bg[0], cam->bg[1], cam->bg[2]}, T = 1.0;
            for (int64_t j = nv - 1; j >= 0; --j) {
                int64_t g = id[j];
                double a = splat_alpha(mean2d, conic, opacity, g, px, py, NULL, NULL, NULL);
                if (!(a >= 1.0 / 255.0)) continue;
                for (int ch = 0; ch < 3; ++ch) C[ch] = a * rgb[3 * g + ch] + (1.0 - a) * C[ch];
                T *= 1.0 - a;
            }
            int64_t pix = (int64_t)v * cam->width + u;
            for (int ch = 0; ch < 3; ++ch) image[3 * pix + ch] = C[ch];
            t_final[pix] = T;
        }
    free(k); free(id);
}

/* ------------------------------------------------------- loss + gradient */

static uint64_t fnv(uint64_t h, uint64_t v) { h ^= v; h *= 1099511628211ull; return h; }

/* L = 1/2 sum (C - target)^2 over the image rendered by the pipeline above
 * (canonical decisions, tile lists from the canonical rects), and, when
 * grads are requested, its analytic gradient w.r.t. means[3], log_scales[3],
 * quats[4], logits[1] and sh[16][3] (the paper has no backward; §1 notes the
 * representation is differentiable). Conventions at the kinks: gradient 0
 * through a clamped 0.99 alpha, a clamped Jacobian ratio and a clamped-at-0
 * colour channel; culled splats and skipped pairs contribute nothing.
 * *fingerprint hashes every discrete decision (culls, per-pair 1/255 tests,
 * clamps) so that finite differences can skip entries whose step changes one.
 * image may be NULL. Returns L. */
double or_loss_grad(int64_t n, const double *means, const double *log_scales,
                    const double *quats, const double *logits, const double *sh,
                    const or_camera *cam, const or_config *cfg, const double *target,
                    double *image_out, double *d_means, double *d_log_scales, double *d_quats,
                    double *d_logits, double *d_sh, uint64_t *fingerprint)
{
    const int TS = cfg->tile, TX = tiles_x(cam, cfg), TY = tiles_y(cam, cfg);
    const int64_t ntiles = (int64_t)TX * TY;
    size_t nn = (size_t)(n > 0 ? n : 1);
    double *mean2d = calloc(nn * 2, 8), *cov2d = calloc(nn * 3, 8), *conic = calloc(nn * 3, 8);
    double *rgb = calloc(nn * 3, 8), *opac = calloc(nn, 8), *ext = calloc(nn * 2, 8);
    float *depth = calloc(nn, 4);
    int32_t *rect = calloc(nn * 4, 4), *rexp = calloc(nn * 4, 4), *touched = calloc(nn, 4), *reason = calloc(nn, 4);
    uint8_t *amb = calloc(nn, 1);
    or_preprocess(n, means, log_scales, quats, logits, sh, cam, cfg, mean2d, cov2d, conic, depth,
                  rgb, opac, ext, rect, rexp, touched, reason, amb);
    int64_t *offs = calloc(nn + 1, 8);
    int64_t K = or_emit_keys(n, rect, depth, TX, NULL, NULL, offs);
    uint64_t *keys = calloc((size_t)(K > 0 ? K : 1), 8);
    uint32_t *vals = calloc((size_t)(K > 0 ? K : 1), 4);
    or_emit_keys(n, rect, depth, TX, keys, vals, offs);
    or_sort_pairs(K, keys, vals);
    int64_t *ranges = calloc((size_t)ntiles * 2, 8);
    or_tile_ranges(K, keys, ntiles, ranges);

    uint64_t fp = 1469598103934665603ull;
    {
        /* discrete states outside the blend: cull reasons, the Jacobian clamp
         * and the colour clamp of each visible splat */
        const double *V = cam->viewmat;
        const double limx = cfg->guard * 0.5 * cam->width / cam->fx, limy = cfg->guard * 0.5 * cam->height / cam->fy;
        for (int64_t i = 0; i < n; ++i) {
            fp = fnv(fp, (uint64_t)reason[i]);
            if (touched[i] == 0) continue;
            const double *X = means + 3 * i;
            double t[3];
            for (int a = 0; a < 3; ++a) t[a] = V[4 * a] * X[0] + V[4 * a + 1] * X[1] + V[4 * a + 2] * X[2] + V[4 * a + 3];
            double rx = t[0] / t[2], ry = t[1] / t[2];
            uint64_t cl = (uint64_t)(rx < -limx || rx > limx) | ((uint64_t)(ry < -limy || ry > limy) << 1);
            for (int ch = 0; ch < 3; ++ch) cl |= (uint64_t)(rgb[3 * i + ch] > 0.0) << (2 + ch);
            fp = fnv(fp, cl);
        }
    }

    /* per-Gaussian accumulators of dL/d(mean2d, conic a b c, sigma, rgb) */
    double *g_m = calloc(nn * 2, 8), *g_q = calloc(nn * 3, 8), *g_s = calloc(nn, 8), *g_c = calloc(nn * 3, 8);
    int64_t maxlist = 0;
    for (int64_t t = 0; t < ntiles; ++t) if (ranges[2 * t + 1] - ranges[2 * t] > maxlist) maxlist = ranges[2 * t + 1] - ranges[2 * t];
    int64_t *lg = malloc((size_t)(maxlist + 1) * 8);
    double *la = malloc((size_t)(maxlist + 1) * 8), *lG = malloc((size_t)(maxlist + 1) * 8), *lT = malloc((size_t)(maxlist + 1) * 8);
    double *ldx = malloc((size_t)(maxlist + 1) * 8), *ldy = malloc((size_t)(maxlist + 1) * 8);
    double loss = 0.0;
    int want = d_means != NULL;

    for (int64_t t = 0; t < ntiles; ++t) {
        int tx = (int)(t % TX), ty = (int)(t / TX);
        for (int v = ty * TS; v < (ty + 1) * TS && v < cam->height; ++v)
            for (int u = tx * TS; u < (tx + 1) * TS && u < cam->width; ++u) {
                double px = u + 0.5, py = v + 0.5;
                double C[3] = {0, 0, 0}, T = 1.0;
                int64_t m = 0;
                for (int64_t j = ranges[2 * t]; j < ranges[2 * t + 1]; ++j) {
                    int64_t g = vals[j];
                    double G, dx, dy;
                    double a = splat_alpha(mean2d, conic, opac, g, px, py, &G, &dx, &dy);
                    int keep = a >= 1.0 / 255.0;
                    if (!keep) continue;
                    fp = fnv(fp, ((uint64_t)g << 1) | (uint64_t)(opac[g] * G >= 0.99));
                    lg[m] = g; la[m] = a; lG[m] = G; lT[m] = T; ldx[m] = dx; ldy[m] = dy; ++m;
                    for (int ch = 0; ch < 3; ++ch) C[ch] += rgb[3 * g + ch] * a * T;
                    T *= 1.0 - a;
                }
                int64_t pix = (int64_t)v * cam->width + u;
                double dC[3];
                for (int ch = 0; ch < 3; ++ch) {
                    double out = C[ch] + T * cam->bg[ch];
                    if (image_out) image_out[3 * pix + ch] = out;
                    dC[ch] = out - target[3 * pix + ch];
                    loss += 0.5 * dC[ch] * dC[ch];
                }
                if (!want) continue;
                /* Reverse sweep: B = colour of everything behind splat i,
                 * normalised by T_{i+1}; dC/da_i = T_i (c_i - B_i). */
                double B[3] = {cam->bg[0], cam->bg[1], cam->bg[2]};
                for (int64_t k = m - 1; k >= 0; --k) {
                    int64_t g = lg[k];
                    double a = la[k], Ti = lT[k];
                    double dLda = 0.0;
                    for (int ch = 0; ch < 3; ++ch) {
                        g_c[3 * g + ch] += a * Ti * dC[ch];
                        dLda += Ti * (rgb[3 * g + ch] - B[ch]) * dC[ch];
                        B[ch] = a * rgb[3 * g + ch] + (1.0 - a) * B[ch];
                    }
                    if (opac[g] * lG[k] >= 0.99) continue; /* clamped alpha */
                    g_s[g] += lG[k] * dLda;
                    double dLdp = a * dLda; /* d a / d power = a, power = -q/2 */
                    const double *Q = conic + 3 * g;
                    double dx = ldx[k], dy = ldy[k];
                    /* power = -1/2 (Qa dx^2 + 2 Qb dx dy + Qc dy^2), d = p - m */
                    g_m[2 * g] += dLdp * (Q[0] * dx + Q[1] * dy);
                    g_m[2 * g + 1] += dLdp * (Q[1] * dx + Q[2] * dy);
                    g_q[3 * g] += dLdp * (-0.5 * dx * dx);
                    g_q[3 * g + 1] += dLdp * (-dx * dy);
                    g_q[3 * g + 2] += dLdp * (-0.5 * dy * dy);
                }
            }
    }

    if (want) {
        const double *V = cam->viewmat;
        double Rv[3][3] = {{V[0], V[1], V[2]}, {V[4], V[5], V[6]}, {V[8], V[9], V[10]}};
        double tv[3] = {V[3], V[7], V[11]};
        double campos[3];
        for (int i = 0; i < 3; ++i) campos[i] = -(Rv[0][i] * tv[0] + Rv[1][i] * tv[1] + Rv[2][i] * tv[2]);
        const double limx = cfg->guard * 0.5 * cam->width / cam->fx, limy = cfg->guard * 0.5 * cam->height / cam->fy;
        for (int64_t i = 0; i < n; ++i) {
            double *dm = d_means + 3 * i, *dl = d_log_scales + 3 * i, *dq = d_quats + 4 * i, *dsh = d_sh + 48 * i;
            memset(dm, 0, 24); memset(dl, 0, 24); memset(dq, 0, 32); memset(dsh, 0, 48 * 8);
            d_logits[i] = 0.0;
            if (touched[i] == 0) continue;
            const double *X = means + 3 * i, *q0 = quats + 4 * i;
            double sigma = opac[i];
            d_logits[i] = g_s[i] * sigma * (1.0 - sigma);

            /* colour: c = max(0, sum Y k + 1/2) */
            double dir0[3] = {X[0] - campos[0], X[1] - campos[1], X[2] - campos[2]};
            double dn = sqrt(dir0[0] * dir0[0] + dir0[1] * dir0[1] + dir0[2] * dir0[2]);
            double dir[3] = {dir0[0] / dn, dir0[1] / dn, dir0[2] / dn};
            double Y[16], dY[16][3];
            or_sh_basis_cart(dir, Y, dY);
            double gdir[3] = {0, 0, 0};
            for (int ch = 0; ch < 3; ++ch) {
                double val = 0.5;
                for (int k = 0; k < 16; ++k) val += Y[k] * sh[(16 * i + k) * 3 + ch];
                if (!(val > 0.0)) continue;
                double gc = g_c[3 * i + ch];
                for (int k = 0; k < 16; ++k) {
                    dsh[3 * k + ch] = Y[k] * gc;
                    for (int a = 0; a < 3; ++a) gdir[a] += sh[(16 * i + k) * 3 + ch] * dY[k][a] * gc;
                }
            }
            /* d = v / |v|: dL/dv = (I - d d^T) dL/dd / |v| */
            double dd = gdir[0] * dir[0] + gdir[1] * dir[1] + gdir[2] * dir[2];
            for (int a = 0; a < 3; ++a) dm[a] += (gdir[a] - dd * dir[a]) / dn;

            /* forward quantities again */
            double qn = sqrt(q0[0] * q0[0] + q0[1] * q0[1] + q0[2] * q0[2] + q0[3] * q0[3]);
            double q[4] = {q0[0] / qn, q0[1] / qn, q0[2] / qn, q0[3] / qn};
            double R[3][3];
            quat_to_rot(q, R);
            double s[3] = {exp(log_scales[3 * i]), exp(log_scales[3 * i + 1]), exp(log_scales[3 * i + 2])};
            double M[3][3], Sig[3][3];
            for (int a = 0; a < 3; ++a) for (int b = 0; b < 3; ++b) M[a][b] = R[a][b] * s[b];
            for (int a = 0; a < 3; ++a) for (int b = 0; b < 3; ++b) {
                double acc = 0; for (int k = 0; k < 3; ++k) acc += M[a][k] * M[b][k]; Sig[a][b] = acc;
            }
            double t[3];
            for (int a = 0; a < 3; ++a) t[a] = Rv[a][0] * X[0] + Rv[a][1] * X[1] + Rv[a][2] * X[2] + tv[a];
            double rx = t[0] / t[2], ry = t[1] / t[2];
            int clx = 0, cly = 0;
            if (rx < -limx) { rx = -limx; clx = 1; }
            if (rx > limx) { rx = limx; clx = 1; }
            if (ry < -limy) { ry = -limy; cly = 1; }
            if (ry > limy) { ry = limy; cly = 1; }
            double fx = cam->fx, fy = cam->fy, tz = t[2];
            double J[2][3] = {{fx / tz, 0.0, -fx * rx / tz}, {0.0, fy / tz, -fy * ry / tz}};
            double Tm[2][3];
            for (int a = 0; a < 2; ++a) for (int b = 0; b < 3; ++b)
                Tm[a][b] = J[a][0] * Rv[0][b] + J[a][1] * Rv[1][b] + J[a][2] * Rv[2][b];

            /* conic = inverse of Sigma' = [[p, r], [r, s']] */
            double p = cov2d[3 * i], r = cov2d[3 * i + 1], sp = cov2d[3 * i + 2];
            double D = p * sp - r * r, D2 = D * D;
            double ga = g_q[3 * i], gb = g_q[3 * i + 1], gc2 = g_q[3 * i + 2];
            /* a = s'/D, b = -r/D, c = p/D */
            double gp = ga * (-sp * sp / D2) + gb * (r * sp / D2) + gc2 * (1.0 / D - p * sp / D2);
            double gs = ga * (1.0 / D - sp * p / D2) + gb * (r * p / D2) + gc2 * (-p * p / D2);
            double gr = ga * (2.0 * r * sp / D2) + gb * (-1.0 / D - 2.0 * r * r / D2) + gc2 * (2.0 * r * p / D2);
            /* symmetric dL/dSigma' */
            double G2[2][2] = {{gp, 0.5 * gr}, {0.5 * gr, gs}};
            /* Sigma' = Tm Sigma Tm^T (+ dilation): dL/dSigma = Tm^T G2 Tm, dL/dTm = 2 G2 Tm Sigma */
            double GS[3][3];
            for (int a = 0; a < 3; ++a) for (int b = 0; b < 3; ++b) {
                double acc = 0;
                for (int k = 0; k < 2; ++k) for (int l = 0; l < 2; ++l) acc += Tm[k][a] * G2[k][l] * Tm[l][b];
                GS[a][b] = acc;
            }
            double GT[2][3];
            for (int a = 0; a < 2; ++a) for (int b = 0; b < 3; ++b) {
                double acc = 0;
                for (int k = 0; k < 2; ++k) for (int l = 0; l < 3; ++l) acc += 2.0 * G2[a][k] * Tm[k][l] * Sig[l][b];
                GT[a][b] = acc;
            }
            /* Tm = J Rv: dL/dJ = GT Rv^T */
            double GJ[2][3];
            for (int a = 0; a < 2; ++a) for (int b = 0; b < 3; ++b)
                GJ[a][b] = GT[a][0] * Rv[b][0] + GT[a][1] * Rv[b][1] + GT[a][2] * Rv[b][2];
            /* J entries as functions of t */
            double gt[3] = {0, 0, 0};
            gt[2] += GJ[0][0] * (-fx / (tz * tz)) + GJ[1][1] * (-fy / (tz * tz));
            /* J02 = -fx rx / tz with rx = tx/tz unless clamped */
            if (!clx) { gt[0] += GJ[0][2] * (-fx / (tz * tz)); gt[2] += GJ[0][2] * (2.0 * fx * rx / (tz * tz)); }
            else gt[2] += GJ[0][2] * (fx * rx / (tz * tz));
            if (!cly) { gt[1] += GJ[1][2] * (-fy / (tz * tz)); gt[2] += GJ[1][2] * (2.0 * fy * ry / (tz * tz)); }
            else gt[2] += GJ[1][2] * (fy * ry / (tz * tz));
            /* mean2d = (fx tx/tz + cx, fy ty/tz + cy) */
            double gmx = g_m[2 * i], gmy = g_m[2 * i + 1];
            gt[0] += gmx * fx / tz;
            gt[1] += gmy * fy / tz;
            gt[2] += -gmx * fx * t[0] / (tz * tz) - gmy * fy * t[1] / (tz * tz);
            for (int a = 0; a < 3; ++a) dm[a] += Rv[0][a] * gt[0] + Rv[1][a] * gt[1] + Rv[2][a] * gt[2];

            /* Sigma = M M^T, M = R S: dL/dM = 2 GS M */
            double GM[3][3];
            for (int a = 0; a < 3; ++a) for (int b = 0; b < 3; ++b) {
                double acc = 0; for (int k = 0; k < 3; ++k) acc += 2.0 * GS[a][k] * M[k][b]; GM[a][b] = acc;
            }
            double GR[3][3];
            for (int b = 0; b < 3; ++b) {
                double gsb = 0;
                for (int a = 0; a < 3; ++a) { gsb += GM[a][b] * R[a][b]; GR[a][b] = GM[a][b] * s[b]; }
                dl[b] = gsb * s[b];
            }
            double w = q[0], x = q[1], y = q[2], z = q[3];
            double gq[4];
            gq[0] = 2 * (-z * GR[0][1] + y * GR[0][2] + z * GR[1][0] - x * GR[1][2] - y * GR[2][0] + x * GR[2][1]);
            gq[1] = 2 * (y * GR[0][1] + z * GR[0][2] + y * GR[1][0] - 2 * x * GR[1][1] - w * GR[1][2] + z * GR[2][0] + w * GR[2][1] - 2 * x * GR[2][2]);
            gq[2] = 2 * (-2 * y * GR[0][0] + x * GR[0][1] + w * GR[0][2] + x * GR[1][0] + z * GR[1][2] - w * GR[2][0] + z * GR[2][1] - 2 * y * GR[2][2]);
            gq[3] = 2 * (-2 * z * GR[0][0] - w * GR[0][1] + x * GR[0][2] + w * GR[1][0] - 2 * z * GR[1][1] + y * GR[1][2] + x * GR[2][0] + y * GR[2][1]);
            /* q_hat = q / |q|: dL/dq = (I - q_hat q_hat^T) dL/dq_hat / |q| */
            double qd = gq[0] * q[0] + gq[1] * q[1] + gq[2] * q[2] + gq[3] * q[3];
            for (int a = 0; a < 4; ++a) dq[a] = (gq[a] - qd * q[a]) / qn;
        }
    }
    if (fingerprint) *fingerprint = fp;
    free(mean2d); free(cov2d); free(conic); free(rgb); free(opac); free(ext); free(depth);
    free(rect); free(rexp); free(touched); free(reason); free(amb); free(offs); free(keys); free(vals);
    free(ranges); free(g_m); free(g_q); free(g_s); free(g_c); free(lg); free(la); free(lG); free(lT);
    free(ldx); free(ldy);
    return loss;
}
