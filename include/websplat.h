/*
 * websplat.h -- C ABI of the GB300 (sm_103a) 3D Gaussian Splatting render
 * path studied in "WebSplatter" (arXiv 2602.03207).
 *
 * A frame is four calls on one CUDA stream, in this order:
 *   ws_preprocess  -> ws_cull -> ws_sort -> ws_rasterize
 * and, for training, ws_rasterize_backward after ws_rasterize.
 *
 * Conventions shared by every entry point
 *   - The caller owns all memory. The library never allocates or frees
 *     device memory; scratch lives in a caller-provided workspace of
 *     ws_workspace_bytes() bytes. Every pointer argument named "device" is
 *     a CUDA device pointer; every struct pointer is a host pointer read
 *     before the call returns.
 *   - Device pointers must be 16-byte aligned (vector loads); a misaligned
 *     pointer returns WS_ERR_INVALID_ARG.
 *   - All work is enqueued asynchronously on `stream` (a cudaStream_t; NULL
 *     is the legacy default stream). No call synchronises the host, so a
 *     whole frame can be captured into a CUDA graph.
 *   - Argument errors are detected on the host before any launch and
 *     returned synchronously (WS_ERR_INVALID_ARG / WS_ERR_UNSUPPORTED); a
 *     launch failure returns WS_ERR_CUDA. Data-dependent errors (more keys
 *     than key_capacity) are recorded in a status word inside the workspace
 *     and read with ws_read_status() after the stream has been synchronised.
 *   - n = 0 and an empty key list are valid; the image is then the
 *     background colour.
 *
 * Layouts (all float32, C-contiguous, Gaussian-major):
 *   means[n][3] world position; log_scales[n][3] log of the per-axis
 *   standard deviations; quats[n][4] rotation quaternion (w, x, y, z), any
 *   non-zero norm; opacity_logits[n]; sh[n][16][3] degree-3 spherical
 *   harmonic coefficients, coefficient-major (index l*l + l + m, real SH
 *   with the Condon-Shortley phase, i.e. the 3DGS PLY convention).
 *
 * Splat record (written by ws_preprocess, read by the blends): per Gaussian
 * WS_SPLAT_FLOATS = 12 float32, 48 bytes, so one gather of a splat touches
 * two 32-byte memory sectors:
 *   [0] x_hi [1] y_hi [2] x_lo [3] y_lo  projected centre as the unevaluated
 *        double-float sum (x_hi + x_lo, y_hi + y_lo) in pixels; x_hi alone
 *        is the float32-rounded centre
 *   [4] a [5] b [6] c                    conic Sigma'^{-1} = [[a, b], [b, c]]
 *   [7] sigma                            opacity
 *   [8] r [9] g [10] b                   colour
 *   [11] t                               tan(theta / 2), theta in [-pi/2, pi/2]
 *        the angle of the major axis of Sigma' = conic^{-1} (0 for a circle);
 *        the backward sums each pair's conic derivatives in the basis
 *        e1 = ((1 - t^2), 2 t) / (1 + t^2), e2 = e1 turned by +90 degrees
 * A culled Gaussian's record is all zeros.
 */
#ifndef WEBSPLAT_H
#define WEBSPLAT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t ws_status;
#define WS_OK 0
#define WS_ERR_INVALID_ARG 1
#define WS_ERR_CUDA 2
#define WS_ERR_CAPACITY 3
#define WS_ERR_TIMEOUT 4
#define WS_ERR_UNSUPPORTED 5

#define WS_ABI_VERSION 2

/* Status bits written to the device status word. */
#define WS_FLAG_CAPACITY 1u /* more (tile, splat) pairs than key_capacity */
#define WS_FLAG_TIMEOUT 2u  /* a bounded wait ran out (look-back sort only) */

#define WS_SPLAT_FLOATS 12 /* floats per splat record (see the layout above) */

/* Pinhole camera (§3.2 projects each centre and covariance to the image).
 * viewmat: row-major 3x4 [R | t] world -> camera, OpenCV axes (x right,
 * y down, z forward). Pixel u covers [u, u+1), so its centre is u + 1/2.
 * Splats with float32 view depth <= znear are culled. bg: background RGB. */
typedef struct ws_camera {
    float viewmat[12];
    float fx, fy, cx, cy;
    int32_t width, height;
    float znear;
    float bg[3];
} ws_camera;

/* Frame configuration.
 *   tile        tile side in pixels: 8, 16 or 32
 *   digit_bits  radix-sort digit width: 4..8 (ws_sort)
 *   dilation    px^2 added to the diagonal of the projected covariance (0.3)
 *   guard       frustum guard factor of the EWA Jacobian clamp (1.3)
 *   flags       WS_CFG_* bits below                                        */
typedef struct ws_config {
    int32_t tile;
    int32_t digit_bits;
    float dilation;
    float guard;
    uint32_t flags;
} ws_config;

#define WS_CFG_NO_OPACITY_CULL 1u /* ablation: keep splats with sigma < 1/255 */
#define WS_CFG_NO_AABB_CULL 2u    /* ablation: keep splats whose box misses the viewport */
#define WS_CFG_SORT_LOOKBACK 4u   /* ws_sort: single-sweep decoupled look-back variant */
#define WS_CFG_FIXED_RADIUS 8u    /* ablation: every splat's box as at sigma = 1 (no opacity-aware extent) */
#define WS_CFG_SORT_SEGMENTED 16u /* ws_sort: partition by bits [31, end) then sort each segment on chip */
#define WS_CFG_PERSISTENT 32u     /* ws_render_train_l2_batch: one persistent grid over every (view, tile) */
#define WS_CFG_RANGES_GIVEN 64u   /* rasterize / train calls: `ranges` already holds the tile ranges (ws_sort_tiles) */
#define WS_CFG_BOX_MASKS 128u     /* backward / train calls: visit every 4x4 sub-block of a splat's bounding box,
                                     not only those that its ellipse meets (same results; an ablation and a check) */

/* Library ABI version (WS_ABI_VERSION of the build). */
int32_t ws_abi_version(void);

/* Human-readable name of a status code (static string). */
const char *ws_status_string(ws_status s);

/* Bytes of workspace the calls below need for n Gaussians, at most
 * key_capacity (tile, splat) pairs, this camera's tile grid and this
 * configuration. Returns 0 for invalid arguments. */
size_t ws_workspace_bytes(int64_t n, int64_t key_capacity, const ws_camera *cam,
                          const ws_config *cfg);

/* Pre-processing stage (§3.2, with §2.1's covariance and colour and §3.4's
 * opacity culling and opacity-aware extent). One thread per Gaussian:
 *   sigma = 1/(1+exp(-logit)); culled if sigma < 1/255 (decided exactly as
 *   logit < -ln 254), if the quaternion is zero, or if the float32 view
 *   depth ((r20 x + r21 y) + r22 z) + t2, evaluated with each operation
 *   rounded, is <= znear;
 *   Sigma = R(q) diag(exp(2 log_scale)) R(q)^T; Sigma' = J W Sigma W^T J^T
 *   + dilation I with the EWA Jacobian J (t_x/t_z, t_y/t_z clamped to the
 *   guard band inside J); conic = Sigma'^{-1};
 *   extent e = sqrt(2 ln(255 sigma) diag(Sigma')) -- the box of the ellipse
 *   where sigma exp(-q/2) >= 1/255 (§3.4's cutoff, read with r^2 = q/2);
 *   culled if [m - e, m + e] misses [0, W) x [0, H) (§3.2 AABB culling);
 *   rgb = max(0, sum_lm sh_lm Y_lm(d) + 1/2), d = normalise(X - camera).
 * Inputs: the Gaussian arrays (device, layouts above).
 * Outputs (device, caller-allocated, n entries each):
 *   splats[n][12] the splat record above (centre, conic, sigma, colour)
 *   depth[n]      float32 view depth (written for every Gaussian)
 *   rect[n][4]    uint16 tile rectangle x0, y0, x1, y1 (inclusive)
 *   tiles_touched[n]  uint32 tiles in rect; 0 means culled
 * Every entry is written; a culled Gaussian gets tiles_touched = 0 and
 * zeros in its splat record and rect. */
ws_status ws_preprocess(int64_t n, const float *means, const float *log_scales,
                        const float *quats, const float *opacity_logits, const float *sh,
                        const ws_camera *cam, const ws_config *cfg, float *splats, float *depth,
                        uint16_t *rect, uint32_t *tiles_touched, void *stream);

/* Compaction of the surviving splats into the <tile, splat> pair list
 * (§3.2 compacts the survivors of culling into a buffer; §3.4 describes
 * the tile-based pair list this path uses). A wait-free two-level scan
 * (one dispatch per level, no inter-block waiting, no global atomics) of
 * tiles_touched gives
 *   offsets[i] = sum_{j<i} tiles_touched[j]   (device, n + 1 entries,
 *                offsets[n] = total pairs),
 * and every visible Gaussian i writes, for each tile (tx, ty) of its rect in
 * row-major order, at slot offsets[i] + k:
 *   keys[slot] = ((ty * tiles_x + tx) << 31) | float32 bits of depth[i]
 *   vals[slot] = i
 * (the depth is positive, so its sign bit is 0 and key order is (tile,
 * depth) order). num_keys (device, one uint32) receives min(total,
 * key_capacity); pairs past key_capacity are dropped and WS_FLAG_CAPACITY
 * is raised. The pair total is accumulated in 64 bits: a frame may cover
 * more than 2^32 pairs, and offsets are then stored saturated at
 * 2^32 - 1 (every such slot lies past the capacity). Clears the workspace
 * status word first. key_capacity must be < 2^31. */
ws_status ws_cull(int64_t n, const uint32_t *tiles_touched, const uint16_t *rect,
                  const float *depth, const ws_camera *cam, const ws_config *cfg,
                  uint32_t *offsets, uint64_t *keys, uint32_t *vals, int64_t key_capacity,
                  uint32_t *num_keys, void *workspace, void *stream);

/* Stable LSD radix sort of (keys, vals) by key bits [begin_bit, end_bit)
 * (§3.3.2). Each pass of cfg->digit_bits bits is three dispatches:
 * per-block digit histograms, a scan of the digit-major histogram matrix
 * giving base_d + prefix_wg for every (digit, block), and a stable scatter
 * to pos = base_d + prefix_wg + rank_local. No block ever waits for
 * another and there are no global atomics, so the result does not depend
 * on scheduling. The key count is read from num_keys (device) so the
 * launch needs no host synchronisation; key_capacity bounds the grids.
 * *num_keys must not exceed key_capacity; a larger count is clamped to
 * key_capacity on the device (the first key_capacity pairs are sorted and
 * nothing past the buffers or the scratch is written).
 * keys_alt / vals_alt (device, key_capacity entries) are the ping-pong
 * buffers. *result_in_alt (host) is set to 1 when the sorted data ends in
 * the _alt buffers (odd pass count), else 0. begin_bit < end_bit <= 64. */
ws_status ws_sort(const uint32_t *num_keys, int64_t key_capacity, int32_t begin_bit,
                  int32_t end_bit, uint64_t *keys, uint32_t *vals, uint64_t *keys_alt,
                  uint32_t *vals_alt, const ws_config *cfg, void *workspace,
                  int32_t *result_in_alt, void *stream);

/* With cfg->flags & WS_CFG_SORT_LOOKBACK (digit_bits 4..9), ws_sort runs a
 * single-sweep variant of the same sort: one read of the keys counts the
 * digits of every pass, then each pass is one kernel over a co-resident
 * persistent grid in which every block publishes its per-digit counts and
 * obtains prefix_wg by looking back over its predecessors (decoupled
 * look-back; release/acquire stores and loads, no read-modify-write
 * atomics). Its result is bit-identical to the default; only progress
 * depends on scheduling, and every wait is bounded (about a second): a wait
 * that runs out raises WS_FLAG_TIMEOUT in the workspace status word, the
 * other blocks stop, nothing is written out of bounds and the call returns
 * (the sorted output is then invalid). The paper avoids such inter-block
 * waiting (§3.3.1); this variant is offered for comparison. */

/* With cfg->flags & WS_CFG_SORT_SEGMENTED (and not WS_CFG_SORT_LOOKBACK),
 * ws_sort treats bits [31, end_bit) of each key as a segment id (the tile of
 * a (tile << 31 | depth) key) and bits [begin_bit, 31) as its sub-key. It
 * partitions the pairs by segment with the wait-free passes above, finds
 * every segment's first position, and sorts each segment by its sub-key on
 * chip (a warp per segment of at most 256 keys, a block otherwise). The
 * partition uses as few passes as digits of at most cfg->digit_bits bits
 * allow. The output, ties included, is bit-identical to the default, with
 * fewer passes over the whole key array (13 tile bits: 2 instead of 5 at
 * 9-bit digits).
 * It applies when 0 <= begin_bit < 31 < end_bit <= 55 and the workspace's
 * sort region holds the 2^(end_bit - 31) + 1 segment starts (about one per
 * key of capacity, at most 2^24 + 1); otherwise ws_sort runs the default sort. Segments of more than 2048 keys are sorted by one block
 * through global memory, correct at any size but slower. */

/* The segmented sort of (tile << 31 | depth) keys over bits [0, end_bit)
 * (ws_sort with WS_CFG_SORT_SEGMENTED and begin_bit 0) that also writes the
 * tile ranges the rasterisation needs: ranges[t] = [start, end) of tile t in
 * the sorted list for t < ntiles (start = end for a tile without pairs),
 * found from the segment boundaries the sort computes anyway. Pass
 * WS_CFG_RANGES_GIVEN to the following ws_rasterize (or training call) of the
 * frame so that it takes `ranges` as given instead of scanning the sorted keys
 * again. ranges (device): ntiles uint32 pairs; ntiles <= 2^(end_bit - 31).
 * Returns WS_ERR_UNSUPPORTED where ws_sort would fall back to the full-key
 * passes (end_bit outside 32..55, or a workspace too small for the segment
 * starts); other errors as ws_sort. */
ws_status ws_sort_tiles(const uint32_t *num_keys, int64_t key_capacity, int32_t end_bit, uint64_t *keys,
                        uint32_t *vals, uint64_t *keys_alt, uint32_t *vals_alt, const ws_config *cfg,
                        void *workspace, uint32_t *ranges, int64_t ntiles, int32_t *result_in_alt,
                        void *stream);

/* ws_cull followed by ws_sort_tiles of the frame's keys (end_bit the
 * smallest with 2^(end_bit - 31) >= the tile count, at least 32), with the
 * compaction fused into the sort's first partition pass: instead of writing
 * the pairs in slot order, the compaction writes each one where that pass
 * would put it (the stable partition of the slot-ordered pairs by the low D
 * bits of the tile id, D the first digit of the segmented sort: 7 at 1080p
 * with 16-pixel tiles and 9-bit digits). Per chunk of Gaussians it counts
 * the pairs of each digit from the rectangles, scans each digit's counts
 * over the chunks, and scatters every pair to base_d + (pairs of digit d in
 * earlier chunks) + (its rank among the chunk's pairs of digit d in slot
 * order): no block waits for another, no global atomics. The results --
 * offsets, num_keys, the sorted keys and vals, ranges, *result_in_alt and
 * the status word -- are bit-identical to those of ws_cull and
 * ws_sort_tiles; pass WS_CFG_RANGES_GIVEN to the following rasterisation.
 * When the frame has more pairs than key_capacity the compaction writes the
 * first key_capacity slots in slot order instead (as ws_cull) and
 * WS_FLAG_CAPACITY is raised; the sorted list is then not meaningful, but
 * every entry below num_keys holds a valid pair. The workspace must come
 * from ws_workspace_bytes with the same n. Returns WS_ERR_UNSUPPORTED when
 * ws_sort_tiles would, or when the first digit is wider than 8 bits (take
 * ws_cull and ws_sort_tiles then). Measured on GB300 at 1080p / 1M: no
 * faster than the two calls (the fused emission costs what the emission and
 * the first pass's scatter cost together, and counting the digits from the
 * rectangles what the first pass's histograms cost). */
ws_status ws_cull_sort_tiles(int64_t n, const uint32_t *tiles_touched, const uint16_t *rect, const float *depth,
                             const ws_camera *cam, const ws_config *cfg, uint32_t *offsets, uint64_t *keys,
                             uint32_t *vals, uint64_t *keys_alt, uint32_t *vals_alt, int64_t key_capacity,
                             uint32_t *num_keys, uint32_t *ranges, void *workspace, int32_t *result_in_alt,
                             void *stream);

/* Test hook of the look-back variant: tile `stalled_tile` of the first pass
 * never publishes its counts, so every later tile's bounded wait runs out.
 * Lets a test check that a stalled predecessor ends in WS_FLAG_TIMEOUT and a
 * usable context instead of a hang. Not for production use. */
ws_status ws_sort_test_stalled_tile(const uint32_t *num_keys, int64_t key_capacity, int32_t begin_bit,
                                    int32_t end_bit, uint64_t *keys, uint32_t *vals, uint64_t *keys_alt,
                                    uint32_t *vals_alt, const ws_config *cfg, void *workspace,
                                    int32_t stalled_tile, int32_t *result_in_alt, void *stream);

/* ws_sort without a workspace, for callers that cannot allocate device
 * memory: code running inside an engine that owns every device allocation
 * and hands over only its input and output buffers, or a real-time frame
 * loop that must not call cudaMalloc (which can synchronise the device).
 * The paper has no counterpart; it is the same sort as ws_sort, with the
 * histogram scratch held in a static device array inside the library
 * (4 MiB + 1 KiB, kept by every GPU that loads the library until the process
 * exits). The caller still passes the keys, values and ping-pong buffers.
 * key_capacity must not exceed ws_sort_noalloc_max_keys() (8,388,608);
 * larger values return WS_ERR_INVALID_ARG. digit_bits: 4..8; any other
 * width returns WS_ERR_UNSUPPORTED. *num_keys must not exceed
 * key_capacity; a larger count is clamped to it on the device. Allocates
 * nothing. The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress), so make that first call before any stream
 * capture. All calls on one device share the array: calls that overlap on
 * the GPU (different streams, concurrent graphs) race and must be ordered
 * by the caller. */
int64_t ws_sort_noalloc_max_keys(void);
ws_status ws_sort_noalloc(const uint32_t *num_keys, int64_t key_capacity, int32_t begin_bit,
                          int32_t end_bit, uint64_t *keys, uint32_t *vals, uint64_t *keys_alt,
                          uint32_t *vals_alt, int32_t digit_bits, int32_t *result_in_alt,
                          void *stream);

/* Rasterisation stage (§3.4 with §2.1's compositing), per 16x16 (tile^2)
 * pixel tile, front to back over the tile's depth-sorted list:
 *   a = min(0.99, sigma exp(-q/2)), q = d^T conic d, d = pixel centre -
 *   centre; pairs with a < 1/255 are skipped; C += rgb a T; T *= 1 - a;
 *   image = C + T bg.
 * Inputs: num_keys (device), sorted keys and vals (device), the splat
 * records of ws_preprocess. Outputs (device): ranges[tiles][2] uint32 [start,
 * end) of every tile in the sorted list (start = end for a tile without
 * pairs); image[H][W][3]; t_final[H][W]
 * (final transmittance); n_contrib[H][W] (1 + list position, relative to
 * the tile's start, of the last splat composited; 0 if none). */
ws_status ws_rasterize(const uint32_t *num_keys, const uint64_t *keys, const uint32_t *vals,
                       const float *splats, const ws_camera *cam, const ws_config *cfg,
                       uint32_t *ranges, float *image, float *t_final, uint32_t *n_contrib,
                       void *stream);

/* The device buffers of one frame (all caller-allocated, 16-byte aligned):
 * the scene's arrays (n entries each, the input layouts) and everything the
 * four calls above read and write, sized as those calls state for n
 * Gaussians, key_capacity pairs and the camera's resolution and tile grid;
 * workspace of ws_workspace_bytes(n, key_capacity, cam, cfg) bytes. */
typedef struct ws_frame_buffers {
    float *means, *log_scales, *quats, *opacity_logits, *sh;
    float *splats, *depth;
    uint16_t *rect;
    uint32_t *tiles_touched, *offsets;
    uint64_t *keys, *keys_alt;
    uint32_t *vals, *vals_alt, *num_keys, *ranges;
    float *image, *t_final;
    uint32_t *n_contrib;
    void *workspace;
    int64_t key_capacity;
} ws_frame_buffers;

/* One frame from a scene in host memory to an image in host memory, all
 * enqueued on `stream`: the five scene arrays are copied host -> device into
 * buf (cudaMemcpyAsync), then ws_preprocess, ws_cull, the sort (ws_sort_tiles
 * where the segmented sort applies, else ws_sort) and ws_rasterize run, and
 * the image is copied device -> host into h_image (H x W x 3 float32). The
 * copies are asynchronous only from page-locked host memory; the call never
 * synchronises the host, so read h_image after synchronising the stream, and
 * check the capacity flag with ws_read_status. Errors as the calls it makes. */
ws_status ws_render_frame_host(int64_t n, const float *h_means, const float *h_log_scales, const float *h_quats,
                               const float *h_opacity_logits, const float *h_sh, const ws_camera *cam,
                               const ws_config *cfg, const ws_frame_buffers *buf, float *h_image, void *stream);

/* Packed-record variant of ws_preprocess (§3.2 packs each splat's colour and
 * opacity into one RGBA8 word and its ellipse axes into two words of
 * binary16 halves). Same inputs and the same culling as ws_preprocess; per
 * visible splat it writes instead:
 *   mean2d[n][2]  float32 centre (px)
 *   axes[n][2]    uint32: (v1.x | v1.y << 16), (v2.x | v2.y << 16) as IEEE
 *                 binary16, the major and minor axes sqrt(l) e of Sigma'
 *                 (Sigma' = v1 v1^T + v2 v2^T), rounded to nearest even
 *   rgba[n]       uint32: r | g << 8 | b << 16 | sigma << 24, each
 *                 round(255 clamp(x, 0, 1)) (colours above 1 are clamped)
 * (every entry written, zeros for a culled Gaussian) and depth, rect and
 * tiles_touched as ws_preprocess, with the extent, the
 * viewport test and the tile rectangle computed from the packed sigma and
 * axes. ws_cull and ws_sort take the outputs unchanged; ws_rasterize_packed
 * reads the packed record. Images differ from the float path by the
 * quantisation (at most about 1/255 per channel where no colour exceeds 1).
 * All pointers device, 16-byte aligned; errors as ws_preprocess. */
ws_status ws_preprocess_packed(int64_t n, const float *means, const float *log_scales, const float *quats,
                               const float *opacity_logits, const float *sh, const ws_camera *cam,
                               const ws_config *cfg, float *mean2d, uint32_t *axes, uint32_t *rgba,
                               float *depth, uint16_t *rect, uint32_t *tiles_touched, void *stream);

/* ws_rasterize on the packed record of ws_preprocess_packed: the blend
 * rebuilds Sigma' from the two axes (det = (v1 x v2)^2), inverts it and
 * decodes colour and sigma from the RGBA8 word; everything else (tile
 * ranges, compositing, outputs, errors) is ws_rasterize's. */
ws_status ws_rasterize_packed(const uint32_t *num_keys, const uint64_t *keys, const uint32_t *vals,
                              const float *mean2d, const uint32_t *axes, const uint32_t *rgba,
                              const ws_camera *cam, const ws_config *cfg, uint32_t *ranges, float *image,
                              float *t_final, uint32_t *n_contrib, void *stream);

/* The paper's own render design (§3.3 sort stage, §3.4 rasterisation stage)
 * in CUDA, for comparison with the tile path: the visible splats
 * (tiles_touched > 0) are compacted and sorted by their 32-bit float depth
 * with four stable 8-bit passes; each becomes one quad sized by its opacity
 * (E8: r = sqrt(ln(255 sigma)) along its ellipse axes) carrying the local
 * coordinate p of E9 (p . p = q / 2); the quads are binned to screen tiles in
 * depth order (a stable partition keeps that order per tile) and every tile
 * composites its quads back to front with "over", C = a c + (1 - a) C, from
 * the background. A fragment is a pixel centre with |p_x|, |p_y| <= r;
 * a = min(0.99, sigma e^{-p.p}) and fragments with a < 1/255 are skipped, so
 * the image equals ws_rasterize's within float rounding.
 * Inputs (device): the ws_preprocess outputs (splats, depth,
 * tiles_touched). keys / vals / keys_alt / vals_alt (device,
 * key_capacity entries) hold the (tile, rank) pairs of the binning;
 * num_keys[0] (device) receives their count (WS_FLAG_CAPACITY in the
 * workspace status word when it exceeds key_capacity). Outputs (device):
 * image[H][W][3], t_final[H][W]. workspace: ws_quads_workspace_bytes(n,
 * key_capacity, cam, cfg) bytes, 16-byte aligned; status read with
 * ws_read_status. Errors as ws_rasterize. */
size_t ws_quads_workspace_bytes(int64_t n, int64_t key_capacity, const ws_camera *cam, const ws_config *cfg);
ws_status ws_render_quads(int64_t n, const float *splats, const float *depth, const uint32_t *tiles_touched,
                          const ws_camera *cam,
                          const ws_config *cfg, int64_t key_capacity, uint64_t *keys, uint32_t *vals,
                          uint64_t *keys_alt, uint32_t *vals_alt, uint32_t *num_keys, float *image, float *t_final,
                          void *workspace, void *stream);

/* Backward of the whole frame for a loss L(image): given d_image = dL/dimage
 * (device, [H][W][3]), writes dL/d(means, log_scales, quats, opacity_logits,
 * sh) (device, the input layouts; zero for culled Gaussians). The paper has
 * no backward (§1 only notes that the representation is differentiable);
 * this is the adjoint of the forward defined above, with no gradient
 * through the 0.99 alpha clamp, the Jacobian's guard-band clamp or a colour
 * channel clamped at 0.
 * Deterministic, without float atomics: each tile walks its list back to
 * front from t_final / n_contrib, reduces each pair's 9 partial derivatives
 * (centre 2, conic 3 in the splat's axis basis (record word 11), sigma 1
 * (times sigma), colour 3) inside the block in a fixed order
 * and writes them to the pair's emission slot offsets[g] + k in the
 * workspace; each Gaussian then sums its slots in order and applies the
 * adjoint of its pre-processing. Bitwise reproducible.
 * Inputs: the Gaussians and camera/config of the forward, the ws_preprocess
 * outputs, offsets (ws_cull), the sorted vals (ws_sort), ranges, t_final and
 * n_contrib (ws_rasterize) of the SAME frame, and the key_capacity the
 * workspace was sized with. opacity_logits may be NULL (sigma is read from
 * the splat records). */
ws_status ws_rasterize_backward(int64_t n, const float *means, const float *log_scales,
                                const float *quats, const float *opacity_logits, const float *sh,
                                const ws_camera *cam, const ws_config *cfg, const float *splats,
                                const uint16_t *rect, const uint32_t *offsets,
                                const uint32_t *tiles_touched, const uint32_t *vals,
                                const uint32_t *ranges, const float *t_final, const uint32_t *n_contrib,
                                const float *d_image, int64_t key_capacity, float *d_means,
                                float *d_log_scales, float *d_quats, float *d_opacity_logits,
                                float *d_sh, void *workspace, void *stream);

/* ---------------------------------------------------------------------------
 * Batched views: up to ws_batch_max_views() cameras of one scene rendered
 * (and differentiated) together. Every view's image is bit-identical to the
 * single-view path; the batch reads the scene once instead of once per view.
 * Per-(view, Gaussian) arrays are view-major: entry (v, g) at v * n + g, with
 * the per-Gaussian layouts of the single-view calls (splats[V][n][12],
 * depth[V][n], rect[V][n][4], tiles_touched[V][n], offsets[V * n + 1]).
 * Every entry is written, with
 * zeros for a (view, Gaussian) that is culled, as in ws_preprocess. Tiles
 * are numbered in one global grid: view v's tiles follow those of views
 * 0..v-1, and the keys carry that global tile id (sort bits [0, 31 +
 * ceil(log2 total tiles))). Images are packed: view v's H_v x W_v x 3 floats
 * start after those of views 0..v-1 (likewise t_final and n_contrib).
 * ranges has one [start, end) pair per global tile. The paper renders one
 * view at a time; this batching has no counterpart there. cams is a host
 * array of `views` cameras; cfg applies to every view. */
int32_t ws_batch_max_views(void);
size_t ws_batch_workspace_bytes(int64_t n, int32_t views, const ws_camera *cams, int64_t key_capacity,
                                const ws_config *cfg);
ws_status ws_preprocess_batch(int64_t n, const float *means, const float *log_scales, const float *quats,
                              const float *opacity_logits, const float *sh, int32_t views,
                              const ws_camera *cams, const ws_config *cfg, float *splats, float *depth,
                              uint16_t *rect, uint32_t *tiles_touched, void *stream);
ws_status ws_cull_batch(int64_t n, int32_t views, const ws_camera *cams, const ws_config *cfg,
                        const uint32_t *tiles_touched, const uint16_t *rect, const float *depth,
                        uint32_t *offsets, uint64_t *keys, uint32_t *vals, int64_t key_capacity,
                        uint32_t *num_keys, void *workspace, void *stream);
ws_status ws_rasterize_batch(const uint32_t *num_keys, const uint64_t *keys, const uint32_t *vals, int64_t n,
                             const float *splats, int32_t views, const ws_camera *cams, const ws_config *cfg, uint32_t *ranges,
                             float *image, float *t_final, uint32_t *n_contrib, void *stream);
/* Gradients summed over the views, in view order (deterministic). */
ws_status ws_rasterize_backward_batch(int64_t n, const float *means, const float *log_scales,
                                      const float *quats, const float *sh, int32_t views,
                                      const ws_camera *cams, const ws_config *cfg, const float *splats,
                                      const uint16_t *rect, const uint32_t *offsets,
                                      const uint32_t *tiles_touched, const uint32_t *vals,
                                      const uint32_t *ranges, const float *t_final,
                                      const uint32_t *n_contrib, const float *d_image,
                                      int64_t key_capacity, float *d_means, float *d_log_scales,
                                      float *d_quats, float *d_opacity_logits, float *d_sh,
                                      void *workspace, void *stream);

/* One training step of the L2 loss L = 1/2 ||image - target||^2 after
 * ws_preprocess, ws_cull and ws_sort: the work of ws_rasterize,
 * ws_image_residual and ws_rasterize_backward in two launches. A first kernel
 * takes each tile once: it composites the tile (the image, t_final and
 * n_contrib of ws_rasterize, bit for bit), forms d = image - target for its
 * pixels in registers, and walks the same list back to front writing each
 * pair's partial derivatives to its emission slot (reusing the staged splat
 * records when the tile's list fits one batch of 256); a second sums each
 * Gaussian's records in slot order and applies the pre-processing adjoint.
 * Arguments are those of the three calls it replaces (target (device)
 * [H][W][3]); the gradients equal ws_rasterize_backward's for d_image =
 * image - target bit for bit. The paper has no training step; this fusion
 * has no counterpart there. Errors as ws_rasterize_backward. */
ws_status ws_render_train_l2(int64_t n, const float *means, const float *log_scales, const float *quats,
                             const float *sh, const ws_camera *cam, const ws_config *cfg, const uint32_t *num_keys,
                             const uint64_t *keys, const uint32_t *vals, const float *splats, const uint16_t *rect,
                             const uint32_t *offsets, const uint32_t *tiles_touched, const float *target,
                             int64_t key_capacity, uint32_t *ranges, float *image, float *t_final,
                             uint32_t *n_contrib, float *d_means, float *d_log_scales, float *d_quats,
                             float *d_opacity_logits, float *d_sh, void *workspace, void *stream);

/* ws_render_train_l2 over a batch of views (the layouts of the batched calls
 * above; target packed like the images), gradients summed over the views in
 * view order. With cfg->flags & WS_CFG_PERSISTENT the per-tile kernel is one
 * persistent grid, as many blocks as fit on the GPU at once, block b taking
 * the (view, tile) items b, b + G, b + 2G, ... of the global tile numbering
 * (a static assignment; no block waits on another); otherwise one block per
 * item. Both give the same results bit for bit. */
ws_status ws_render_train_l2_batch(int64_t n, const float *means, const float *log_scales, const float *quats,
                                   const float *sh, int32_t views, const ws_camera *cams, const ws_config *cfg,
                                   const uint32_t *num_keys, const uint64_t *keys, const uint32_t *vals,
                                   const float *splats, const uint16_t *rect, const uint32_t *offsets,
                                   const uint32_t *tiles_touched, const float *target, int64_t key_capacity,
                                   uint32_t *ranges, float *image, float *t_final, uint32_t *n_contrib,
                                   float *d_means, float *d_log_scales, float *d_quats, float *d_opacity_logits,
                                   float *d_sh, void *workspace, void *stream);

/* d_image = image - target over `count` floats (device): the gradient of the
 * L2 loss 1/2 ||image - target||^2 used by the training step. */
ws_status ws_image_residual(int64_t count, const float *image, const float *target, float *d_image,
                            void *stream);

/* Reads (and, if clear != 0, clears) the device status word of a workspace:
 * waits for `stream`, then stores the WS_FLAG_* bits in *flags (host). This
 * is the one call that synchronises the host. */
ws_status ws_read_status(void *workspace, uint32_t *flags, int32_t clear, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* WEBSPLAT_H */
