/*
 * qrender.h -- C ABI of libqrender, a GB300 (sm_103a) implementation of the
 * hot path of Quantile Rendering (Q-Render, arXiv 2512.20927).
 *
 * The paper states the operation as  f~^Q = QuantileRender(G, F, K, I)
 * (Sec. 4.2, Algorithm 1): given 3D Gaussians G, per-Gaussian C-dimensional
 * features F, the number of quantile Gaussians K and the depth-ordered index
 * list I of the Gaussians rasterised at a pixel, return the pixel's rendered
 * feature.  The list I comes from 3D-GS rasterisation: EWA projection of each
 * Gaussian, tiling and a depth sort (Sec. 3).  This library splits that path
 * into calls that can be timed and checked one by one:
 *
 *   qr_project  -> qr_sort -> qr_select -> qr_blend        (Q-Render)
 *   qr_project  -> qr_sort -> qr_dense                     (Eq. 1, V-Render)
 *
 * Conventions shared by every call
 *   - All array pointers are DEVICE pointers owned by the caller unless the
 *     parameter name ends in _host.  The library never allocates device memory
 *     on these paths: scratch lives in a caller-allocated workspace whose size
 *     qr_workspace_bytes() returns.
 *   - Every call is asynchronous on the caller's stream (NULL = the legacy
 *     default stream) and returns a qr_status for what it can check on the
 *     host (arguments, alignment, launch errors).  Conditions found on the
 *     device (intersection capacity exceeded) are written to a status word in
 *     the workspace; qr_frame_status() synchronises the stream and reads it.
 *   - Layouts are row-major.  Gaussian i's parameters are mean[3i..3i+2],
 *     log_scale[3i..3i+2] (natural log of the per-axis standard deviation),
 *     quat[4i..4i+3] = (w, x, y, z) (normalised inside) and opacity[i]
 *     (already activated, in (0, 1)).  Feature row i is feat[i*C .. i*C+C-1].
 *     Pixel p = y * width + x is sampled at (x + 0.5, y + 0.5).
 *   - Feature rows must start on 16-byte boundaries: C % 4 == 0 for FP32,
 *     C % 8 == 0 for BF16, C % 16 == 0 for FP8; feat must be 16-byte aligned.
 *   - Errors never leave partial work queued that reads out of bounds: a call
 *     that returns anything but QR_OK has launched nothing.
 *
 * Thread safety: calls on different workspaces may run concurrently on
 * different streams.  Two calls that use the same workspace race unless they
 * are ordered on one stream.
 */
#ifndef QRENDER_H
#define QRENDER_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Same type as cudaStream_t. */
typedef struct CUstream_st *qr_stream;

typedef enum {
    QR_OK = 0,
    QR_ERR_INVALID_ARG = 1,     /* null pointer, size out of range, bad enum */
    QR_ERR_ALIGNMENT = 2,       /* pointer or row not 16-byte aligned */
    QR_ERR_CAPACITY = 3,        /* more tile-Gaussian intersections than max_isect */
    QR_ERR_CUDA = 4,            /* a CUDA runtime call failed */
    QR_ERR_DEVICE_TIMEOUT = 5,  /* a bounded device-side wait gave up */
    QR_ERR_NOT_SUPPORTED = 6    /* combination not built (e.g. dtype for this call) */
} qr_status;

typedef enum { QR_F32 = 0, QR_BF16 = 1, QR_FP8E4M3 = 2 } qr_dtype;

/* Pinhole camera: camera-space point = R * world + t (x right, y down, z
 * forward); pixel = (fx * x / z + cx, fy * y / z + cy).  Gaussians whose mean
 * has z <= near_plane are culled (Sec. 3 leaves the camera model open). */
typedef struct {
    float R[9];
    float t[3];
    float fx, fy, cx, cy;
    float near_plane;
    int32_t width, height;
} qr_camera;

/* Renderer parameters.  Defaults: qr_default_params(). */
typedef struct {
    int32_t K;          /* quantile Gaussians per pixel, 1..32 (Algorithm 1)           */
    float alpha_min;    /* list membership: alpha' >= alpha_min (1/255)                 */
    float alpha_max;    /* alpha' = min(alpha_max, alpha * G(u)) (0.99)                 */
    float T_min;        /* dense blend stops before T would fall below it (1e-4); 0 = all */
    float dilation;     /* px^2 added to the EWA covariance diagonal (0.3)              */
    int32_t tile_w;     /* screen tile: 16x16 or 8x32 (tile_w * tile_h == 256)          */
    int32_t tile_h;
} qr_params;

/* Host-side descriptor of one frame's workspace.  Filled by qr_frame_init;
 * the caller owns the struct and the workspace it points into.  Fields other
 * than the documented ones are private to the library. */
#define QR_FRAME_SLOTS 24
typedef struct {
    int64_t n;                 /* number of Gaussians                     */
    int64_t max_isect;         /* capacity of the tile-intersection lists */
    qr_camera camera;
    qr_params params;
    int32_t tiles_x, tiles_y;  /* screen tiles                            */
    int32_t sort_blocks;       /* reserved (zero)                         */
    int32_t isect_buf;         /* private                                 */
    void *ws;                  /* device workspace                        */
    size_t ws_bytes;
    size_t off[QR_FRAME_SLOTS];/* private: byte offsets into ws           */
} qr_frame;

/* Device pointers into a frame's workspace, for inspection and tests. */
typedef struct {
    const float *mean2d_hi_lo;   /* [n][4]: projected mean (x_hi, y_hi, x_lo, y_lo); x = x_hi + x_lo   */
    const float *axes;           /* [n][4]: (w1x, w1y, w2x, w2y), conic A = 2 (w1 w1^T + w2 w2^T)        */
    const float *opacity;        /* [n]: alpha of each kept Gaussian                                   */
    const uint32_t *depth_key;   /* [n]: FP32 bit pattern of camera depth; 0xFFFFFFFF when culled      */
    const uint32_t *tile_count;  /* [n]: tiles touched by Gaussian i's footprint                       */
    const uint32_t *kept_gid;    /* [n_kept]: ids of the Gaussians with a footprint, ascending          */
    const uint32_t *kept_offset; /* [n_kept]: first intersection slot of each kept Gaussian             */
    const uint32_t *isect_gid;   /* [n_isect]: per tile, the Gaussian ids in (depth, id) order          */
    const uint32_t *tile_range;  /* [tiles][2]: [begin, end) of each tile in isect_gid                  */
    const uint32_t *counters;    /* [8]: status, n_isect, n_kept, n, n_emitted                         */
} qr_frame_view;

/* ---------------------------------------------------------------- setup */

/* ABI version of this header (incremented on incompatible changes). */
int32_t qr_abi_version(void);

/* Human-readable name of a status code (static string). */
const char *qr_status_string(qr_status s);

/* Fill *p with the defaults listed in qr_params. */
void qr_default_params(qr_params *p);

/* Bytes of workspace a frame of n Gaussians at width x height needs with room
 * for max_isect tile-Gaussian intersections.  0 if an argument is invalid. */
size_t qr_workspace_bytes(int64_t n, int32_t width, int32_t height, const qr_params *params,
                          int64_t max_isect);

/* Lay out a frame in a caller-allocated device workspace ws (256-byte
 * aligned, at least qr_workspace_bytes(...) bytes).  Host only; launches
 * nothing.  QR_ERR_INVALID_ARG on bad sizes or a too small workspace. */
qr_status qr_frame_init(qr_frame *frame, int64_t n, const qr_camera *camera,
                        const qr_params *params, int64_t max_isect, void *ws, size_t ws_bytes);

/* Device pointers of the frame's internal arrays (see qr_frame_view). */
qr_status qr_frame_view_get(const qr_frame *frame, qr_frame_view *view);

/* Synchronise the stream and read the frame's device status word.  Returns
 * QR_ERR_CAPACITY if the intersection lists overflowed (the outputs of
 * qr_sort and everything after it are then zero, not partial), otherwise
 * QR_OK.  n_isect (nullable) receives the number of intersections the frame
 * needed, which is also the capacity to ask for on a retry. */
qr_status qr_frame_status(const qr_frame *frame, qr_stream stream, int64_t *n_isect);

/* ---------------------------------------------------------------- hot path */

/* Sec. 3 (EWA splatting [Zwicker et al.] as used by 3D-GS): per Gaussian,
 * Sigma = R S S^T R^T, Sigma' = J W Sigma W^T J^T + dilation * I with J the
 * Jacobian of the pinhole projection at the camera-space mean, conic
 * A = Sigma'^{-1}, projected mean, camera depth, and the screen tiles its
 * support {u : alpha * exp(-q(u)/2) >= alpha_min} can reach.  Camera-space
 * position, projected mean and conic are computed in compensated
 * (double-FP32) arithmetic, so the stored mean carries a high and low part.
 * Inputs: mean/log_scale [n][3], quat [n][4], opacity [n] (float32, device).
 * Writes only the frame's workspace. */
qr_status qr_project(qr_frame *frame, const float *mean, const float *log_scale,
                     const float *quat, const float *opacity, qr_stream stream);

/* Sec. 3 "tiling strategy" + the depth-ordered list I of Sec. 4.2: bins every
 * kept Gaussian into the screen tiles its footprint touches (load-balanced
 * expansion), and sorts each tile's list by (camera depth, id) in shared
 * memory with a hand-written bitonic network (chunked merge for lists larger
 * than shared memory).  The result -- tile ranges and per-tile id lists -- is
 * the order a sort of 64-bit (tile << 32 | depth) keys would give, with equal
 * depths broken by id.  Overflow of max_isect is reported through
 * qr_frame_status. */
qr_status qr_sort(qr_frame *frame, qr_stream stream);

/* Algorithm 1 (Sec. 4.2), selection half: for every pixel, walk the tile's
 * list front to back with alpha' = min(alpha_max, alpha * exp(-q/2)),
 * skipping alpha' < alpha_min, and keep each Gaussian whose test
 * transmittance T(1 - alpha') crosses the next boundary (K-k)/(K+1) (strict
 * '<'); stop once it falls below 1/(K+1).  Outputs ids [P][K] int32 (depth
 * order, -1 padded), weights [P][K] float32 = T^Q alpha' / (1 - T^Q) (the
 * normalisation of Algorithm 1 folded in; zero padded), counts [P] uint8.
 * P = width * height. */
qr_status qr_select(const qr_frame *frame, int32_t *ids, float *weights, uint8_t *counts,
                    qr_stream stream);

/* The select rules the paper weighs Algorithm 1 against, and App. C's weight
 * form of Algorithm 1, with the outputs of
 * qr_select (ids [P][K] in depth order, -1 padded; weights [P][K]
 * normalised, zero padded; counts [P]), so qr_blend renders any of them.
 *   QR_RULE_QUANTILE:   Algorithm 1 (the same kernel as qr_select).
 *   QR_RULE_TOPK:       top-K, the renderer of Sec. 4.2 and the complexity
 *                       table (O(N log K + KC)): the K largest Eq. 1 weights
 *                       w = T alpha' along the dense walk (alpha' rules and
 *                       T_min stop of qr_dense), equal weights keeping the
 *                       earlier entry; weights divided by the kept sum.
 *   QR_RULE_STRATIFIED: Stratified-K, App. E: pass 1 takes the mean mu and
 *                       standard deviation sigma of the dense walk's
 *                       transmittances; the boundaries
 *                       tau_k = mu + sigma Phi^-1(u_lo + (u_hi - u_lo)(1 - k/(K+1))),
 *                       u_lo = Phi(-mu/sigma), u_hi = Phi((1 - mu)/sigma),
 *                       are equally spaced in the probability of
 *                       N(mu, sigma^2) over [0, 1] (Algorithm 1's
 *                       1 - k/(K+1) with fewer than two blended Gaussians);
 *                       pass 2 is Algorithm 1 with tau_k in place of
 *                       1 - k/(K+1), weights T^Q alpha' / (1 - T^Q).
 *   QR_RULE_RIEMANN:    App. C's right-Riemann reading of Algorithm 1:
 *                       qr_select's ids and counts; each quantile
 *                       Gaussian weighs the number of boundaries
 *                       1 - k/(K+1) its test transmittance crosses,
 *                       divided by the number crossed in all.
 * tau [P][K] float32 (nullable; stratified only) receives each pixel's
 * boundaries.  K <= 32 (frame params). */
typedef enum {
    QR_RULE_QUANTILE = 0,
    QR_RULE_TOPK = 1,
    QR_RULE_STRATIFIED = 2,
    QR_RULE_RIEMANN = 3
} qr_rule;
qr_status qr_select_rule(const qr_frame *frame, qr_rule rule, int32_t *ids, float *weights,
                         uint8_t *counts, float *tau, qr_stream stream);

/* Algorithm 1, blend half ("alpha-blending on quantile Gaussians" +
 * normalisation): out[p] = sum_{j < counts[p]} weights[p][j] * feat[ids[p][j]]
 * with FP32 accumulation.  feat is [n_gauss][C] of dtype; feat_scale [n_gauss]
 * float32 multiplies FP8 rows (NULL otherwise).  out is [P][C] float32.
 * Pixels with counts 0 get zeros.  ids must lie in [0, n_gauss).
 * width > 0 declares the P pixels a row-major image of that width: pixels are
 * then visited in 16x16 screen tiles with 2x2 groups sharing feature rows;
 * width = 0 groups consecutive pixels, whose output rows then form one
 * contiguous run per group (the faster order on GB300, and the one qr_render
 * uses).  Only the summation order (and speed) depends on it. */
qr_status qr_blend(const void *feat, const float *feat_scale, qr_dtype dtype, int32_t C,
                   int64_t n_gauss, const int32_t *ids, const float *weights,
                   const uint8_t *counts, int64_t P, int32_t K, int32_t width, float *out,
                   qr_stream stream);

/* Eq. 1 (V-Render, the dense method the paper compares against):
 * out[p] = sum_i T_i alpha'_i f_i over the pixel's whole list with the same
 * alpha' rules, stopping before a Gaussian whose test transmittance would fall
 * below T_min.  out [P][C] float32; T_final [P] float32 (nullable). */
qr_status qr_dense(const qr_frame *frame, const void *feat, const float *feat_scale,
                   qr_dtype dtype, int32_t C, float *out, float *T_final, qr_stream stream);

/* qr_dense that also counts its work, for measurement: counts [2] device
 * uint64 (zeroed by the call) receive the blended (pixel, Gaussian) pairs --
 * each C multiply-adds of useful work -- and the multiply-adds the kernel
 * executed (rows of 128, 256 or 512 channels; both stay 0 for other widths). */
qr_status qr_dense_work(const qr_frame *frame, const void *feat, const float *feat_scale,
                        qr_dtype dtype, int32_t C, float *out, float *T_final, uint64_t *counts,
                        qr_stream stream);

/* The whole Q-Render forward of one frame: qr_project, qr_sort, qr_select and
 * qr_blend in order on one stream.  ids/weights/counts are kept for a later
 * backward. */
qr_status qr_render(qr_frame *frame, const float *mean, const float *log_scale,
                    const float *quat, const float *opacity, const void *feat,
                    const float *feat_scale, qr_dtype dtype, int32_t C, int32_t *ids,
                    float *weights, uint8_t *counts, float *out, qr_stream stream);

/* End-to-end variant for callers holding HOST arrays: copies the Gaussians
 * and features from host memory (pinned for asynchronous copies) into
 * caller-provided device staging buffers, renders with qr_render, and copies
 * the [P][C] float32 map back into out_host.  dev_inputs must hold
 * 11*n float32 followed (16-byte aligned) by the feature table; dev_outputs
 * must hold the ids/weights/counts/map of qr_render (see qr_render_host_bytes).
 * The call returns once the work is queued; synchronise the stream before
 * reading out_host. */
qr_status qr_render_host_bytes(int64_t n, int32_t width, int32_t height, int32_t K, int32_t C,
                               qr_dtype dtype, size_t *dev_inputs_bytes,
                               size_t *dev_outputs_bytes);
qr_status qr_render_host(qr_frame *frame, const float *mean_host, const float *log_scale_host,
                         const float *quat_host, const float *opacity_host,
                         const void *feat_host, const float *feat_scale_host, qr_dtype dtype,
                         int32_t C, void *dev_inputs, void *dev_outputs, float *out_host,
                         qr_stream stream);

/* ---------------------------------------------------------------- many views */

/* One view of a batch: its frame (already through qr_project and qr_sort),
 * the feature table of its scene, and its outputs (layouts as in qr_select
 * and qr_blend). */
typedef struct {
    const qr_frame *frame;
    const void *feat;
    const float *feat_scale;
    int32_t *ids;
    float *weights;
    uint8_t *counts;
    float *out;
} qr_view;

/* Bytes of device workspace for the descriptors of n_views views. */
size_t qr_batch_workspace_bytes(int32_t n_views);

/* Copy the per-view descriptors into ws (set-up; synchronises the stream so
 * views may be freed afterwards).  All views must share K.  total_tiles
 * receives the number of (view, tile) work items. */
qr_status qr_batch_prepare(const qr_view *views, int32_t n_views, void *ws, size_t ws_bytes,
                           uint32_t *total_tiles, qr_stream stream);

/* Algorithm 1 (selection and blend) for every tile of every prepared view in
 * one persistent launch: CTAs take (view, tile) items from a device counter;
 * in each CTA four warps select a tile's quantile Gaussians into one of two
 * shared-memory buffers while the other warps blend the previously selected
 * tile from the other buffer (same selection arithmetic as qr_select, the
 * same per-channel sums as qr_blend with width > 0; ids/weights/counts are
 * also written).  dtype and C are shared by the batch (rows of 32, 64 or 128
 * sixteen-byte vectors: e.g. 512-D F32 / BF16 / FP8); group = pixels per
 * warp in the blend (4, 2 or 1; 0 = largest allowed by K); chunks = channel
 * slices per feature row for groups of 4, taken by different blend warps
 * (1, 2 or 4 dividing C / 128 and leaving at most 512 channels per slice;
 * 0 = the built-in choice);
 * blend_warps = blend warps per CTA beside the four selection warps (4 or 8;
 * 0 = 8); ctas_per_sm caps the resident CTAs per SM (0 = occupancy limit).
 * Results do not depend on group size or chunks beyond the summation order
 * of a pixel's rows (chunks, blend_warps: not at all).  Capturable in a CUDA
 * graph. */
qr_status qr_render_batch(const void *ws, int32_t n_views, uint32_t total_tiles, qr_dtype dtype,
                          int32_t C, int32_t K, int32_t group, int32_t chunks,
                          int32_t blend_warps, int32_t ctas_per_sm, qr_stream stream);

/* ---------------------------------------------------------------- backward */

/* Backward of Algorithm 1.  The paper states that image-space gradients flow
 * through Q-Render into the per-Gaussian features (Sec. 1, Sec. 4.2) without a
 * formula; with the quantile Gaussians j of a pixel (depth order),
 * a_j = alpha'_j, P_j = prod_{l<j} (1 - a_l), T^Q = P_{m+1}, D = 1 - T^Q and
 * g = dL/dF_p:
 *   dL/df_j   = w_j g                                  (w_j = a_j P_j / D)
 *   dL/da_j   = [P_j s_j - sum_{l>j} a_l P_l s_l / (1-a_j)] / D
 *               - (g.F) T^Q / ((1-a_j) D),             s_l = g . f_l
 *   dL/dalpha = dL/da * exp(-q/2);  dL/d(A00, A01, A11) = dL/da * (-a/2) *
 *               (dx^2, 2 dx dy, dy^2), both zero where alpha' was clamped;
 * the selection itself is piecewise constant and held fixed.
 * frame must still hold the forward's projection and tile lists (qr_project
 * and qr_sort of the same frame), ids/weights/counts its qr_select outputs and
 * feat the table qr_blend used.  grad_out [P][C] float32.  Outputs (all
 * overwritten): grad_feat [n][C] float32 (zero rows for Gaussians no pixel
 * selected), grad_opacity [n] and grad_conic [n][3] (both nullable).  The sum
 * over pixels is deterministic: per-tile partials reduced in a fixed order, no
 * floating-point atomics.  ws: qr_backward_workspace_bytes(frame, C) bytes,
 * 256-byte aligned (about max_isect * C * 4 bytes of partial rows).  The
 * outputs are cleared on a library-owned stream of the current device that is
 * forked from `stream` (event record, wait) and joined back to it within the
 * call, so the call stays ordered on `stream` and can be captured in a CUDA
 * graph. */
size_t qr_backward_workspace_bytes(const qr_frame *frame, int32_t C);
qr_status qr_backward(const qr_frame *frame, const void *feat, const float *feat_scale,
                      qr_dtype dtype, int32_t C, const int32_t *ids, const float *weights,
                      const uint8_t *counts, const float *grad_out, float *grad_feat,
                      float *grad_opacity, float *grad_conic, void *ws, size_t ws_bytes,
                      qr_stream stream);

/* Loss of the differentiation workload (the paper trains with the contrastive
 * Eq. 2 on CLIP targets, which are not available): L = mean over pixels with
 * counts > 0 of 1 - cos(F_p, t_p), cos = F.t / (max(|F|, 1e-8) max(|t|, 1e-8)).
 * feature_map, target [P][C]; loss_out [2] device floats receive (L, 1/n)
 * (they hold integer counters while the call runs on the stream; (0, 1) for
 * P = 0);
 * grad [P][C] receives dL/dF (zero on pixels without quantile Gaussians);
 * scratch [P] floats (overwritten).  Deterministic reduction: the covered
 * pixels are counted with integer atomics and the per-pixel terms are summed
 * over fixed ranges whose sums are added in a fixed order. */
qr_status qr_cosine_loss(const float *feature_map, const float *target, const uint8_t *counts,
                         int64_t P, int32_t C, float *loss_out, float *grad, float *scratch,
                         qr_stream stream);

/* The cosine loss above and the backward above in one call, with the loss's
 * per-pixel pass fused into the backward's: every pixel's dL/dF is formed in
 * registers from its map and target rows, written to grad_map (the upstream
 * gradient of the rest of the backward) and dotted with its quantile
 * Gaussians' features at once, so grad_map is not read back for those dots.
 * Same results as qr_cosine_loss(feature_map, target, mask, ...) followed by
 * qr_backward(..., grad_out = grad_map, ...) up to floating-point summation
 * order.  counts: the forward's quantile counts; mask [P]: pixels in the loss
 * (e.g. the counts themselves); loss_out [2] device floats -> (L, 1/n);
 * grad_map [P][C] -> dL/dF; feature_map, target, grad_map, grad_feat 16-byte
 * aligned; ws: qr_cosine_backward_workspace_bytes(frame, C) bytes, 256-byte
 * aligned (the backward's workspace plus P floats of loss terms). */
size_t qr_cosine_backward_workspace_bytes(const qr_frame *frame, int32_t C);
qr_status qr_cosine_backward(const qr_frame *frame, const void *feat, const float *feat_scale,
                             qr_dtype dtype, int32_t C, const int32_t *ids, const float *weights,
                             const uint8_t *counts, const float *feature_map, const float *target,
                             const uint8_t *mask, float *loss_out, float *grad_map,
                             float *grad_feat, float *grad_opacity, float *grad_conic, void *ws,
                             size_t ws_bytes, qr_stream stream);

/* The training loss of the paper, Eq. 2 (Sec. 4.3): every pixel p of a mask
 * (patch) i = mask_id[p] is pulled towards that mask's CLIP embedding t_i and
 * away from the other masks' embeddings,
 *   L_p = -log( exp(s_i) / sum_{j != i} exp(s_j) ),  s_j = cos(F_p, t_j)
 *       = F.t_j / (max(|F|, 1e-8) max(|t_j|, 1e-8))
 * (the denominator over the other masks j != i, as Eq. 2 prints it), and
 * L = mean of L_p over the pixels with mask_id >= 0 (their count floored at
 * 1).  feature_map [P][C] float32 (the rendered map), targets [M][C] float32
 * (one embedding per mask, any length), mask_id [P] int32 (-1: pixel not in
 * the loss); loss_out [2] device floats -> (L, 1/n) (integer counters while
 * the call runs on the stream); grad [P][C] -> dL/dF (zero rows outside the
 * masks).  2 <= M <= 64; C a multiple of 128 up to 512.  ws: 256-byte
 * aligned, qr_contrastive_workspace_bytes(P, M, C) bytes (unit targets and
 * per-pixel terms).  Deterministic: the terms are summed over fixed ranges
 * added in a fixed order.  QR_ERR_NOT_SUPPORTED for other M or C. */
size_t qr_contrastive_workspace_bytes(int64_t P, int32_t M, int32_t C);
qr_status qr_contrastive_loss(const float *feature_map, const float *targets, int32_t M,
                              int32_t C, const int32_t *mask_id, int64_t P, float *loss_out,
                              float *grad, void *ws, size_t ws_bytes, qr_stream stream);

/* qr_contrastive_loss followed on the stream by qr_backward with its dL/dF
 * (grad_map) as the upstream gradient: one call from the rendered map and
 * the masks' embeddings to the gradients of the features, opacities and
 * conics.  Arguments as in the two calls; ws:
 * qr_contrastive_backward_workspace_bytes(frame, M, C) bytes. */
size_t qr_contrastive_backward_workspace_bytes(const qr_frame *frame, int32_t M, int32_t C);
qr_status qr_contrastive_backward(const qr_frame *frame, const void *feat, const float *feat_scale,
                                  qr_dtype dtype, int32_t C, const int32_t *ids,
                                  const float *weights, const uint8_t *counts,
                                  const float *feature_map, const float *targets, int32_t M,
                                  const int32_t *mask_id, float *loss_out, float *grad_map,
                                  float *grad_feat, float *grad_opacity, float *grad_conic,
                                  void *ws, size_t ws_bytes, qr_stream stream);

/* ---------------------------------------------------------------- relevance */

/* Open-vocabulary relevance (Sec. 5 scores features against text embeddings by
 * cosine similarity): out[p][q] = sum_c map[p][c] * Q[q][c] on the tensor
 * cores (tcgen05, FP32 accumulation in TMEM).  Where the queries fit in shared
 * memory as FP32 (Q * C * 4 bytes plus four 16 KB map stages <= 227 KB) the
 * map is streamed by TMA and multiplied as TF32 (at least 10 mantissa bits);
 * otherwise it is rounded to BF16 on the fly.  feature_map [P][C] float32,
 * queries_bf16 [Q][C] (unit vectors give cosine similarity against
 * unit-normalised features), out [P][Q] float32.  Q in {16, 32, 64, 128}; C a
 * multiple of 64 with the BF16 queries fitting in shared memory (Q * C * 2
 * bytes <= ~190 KB).  status: a device int32 the kernel sets to
 * QR_ERR_DEVICE_TIMEOUT if a bounded wait gives up (it is never cleared by the
 * library; see qr_set_wait_limit). */
qr_status qr_relevance(const float *feature_map, const uint16_t *queries_bf16, int32_t Q, int32_t C,
                       int64_t P, float *out, int32_t *status, qr_stream stream);

/* The blend of Algorithm 1 fused with the relevance product (Sec. 5 scores
 * rendered features against text embeddings): out[p][q] = sum_c F_p[c] Q[q][c]
 * with F_p = sum_{j < counts[p]} weights[p][j] feat[ids[p][j]] (qr_blend's
 * map), without writing the [P][C] map.  Blocks of 128 pixels (16 x 8 on
 * screen when width > 0, consecutive pixels when width = 0) are blended 128
 * channels at a time into shared memory with FP32 accumulation, rounded to
 * BF16 and multiplied on the tensor cores against the BF16 queries with FP32
 * accumulation in TMEM, so out is within 2^-8 sum_c |F_c q_c| of the exact
 * product (like qr_relevance's BF16 kernel).  feat / feat_scale / dtype /
 * ids / weights / counts / P / K / width as in qr_blend (K <= 8);
 * queries_bf16 [Q][C]; out [P][Q] float32.  Q in {16, 32, 64, 128}; C a
 * multiple of 128 with the queries fitting in shared memory (Q * C * 2 bytes
 * plus 90 KB); QR_ERR_NOT_SUPPORTED otherwise.  status as in qr_relevance
 * (QR_ERR_DEVICE_TIMEOUT if a bounded wait gives up). */
qr_status qr_blend_relevance(const void *feat, const float *feat_scale, qr_dtype dtype, int32_t C,
                             int64_t n_gauss, const int32_t *ids, const float *weights,
                             const uint8_t *counts, int64_t P, int32_t K, int32_t width,
                             const uint16_t *queries_bf16, int32_t Q, float *out, int32_t *status,
                             qr_stream stream);

/* ---------------------------------------------------------------- feature storage */

/* Storage formats of the feature table; the paper stores FP32 (Sec. 4).
 * BF16: out[i] = in[i] rounded to nearest even (bit pattern as uint16).
 * count elements, device pointers; asynchronous on stream. */
qr_status qr_quantize_bf16(const float *in, int64_t count, uint16_t *out, qr_stream stream);

/* FP8 E4M3 with one FP32 scale per row: scale[r] = max_c |in[r][c]| / 448
 * (1 for an all-zero row), codes[r][c] = E4M3(in[r][c] / scale[r]) rounded to
 * nearest even and saturated to +-448.  in [rows][C], codes [rows][C],
 * scale [rows].  Decoding is E4M3(code) * scale (qr_blend / qr_dense with
 * QR_FP8E4M3 do it in registers). */
qr_status qr_quantize_fp8(const float *in, int64_t rows, int32_t C, uint8_t *codes,
                          float *scale, qr_stream stream);

/* ---------------------------------------------------------------- allocation-free variant */

/* No counterpart in the paper.  The Q-Render forward of qr_render for callers
 * that may not allocate device memory: a plug-in whose host application owns
 * all device memory through its own pool, a real-time loop in which an
 * allocation could block or fail, or code that prepares everything before a
 * CUDA graph is recorded.  Inputs and outputs are the caller's, with the
 * meaning and layout of qr_render for n Gaussians and the given camera and
 * params; the scratch workspace qr_render would take from the caller is a
 * 16 MiB static device array inside this library instead, which every GPU
 * that loads the library holds until the process exits.
 * Limits: n <= 65,536 Gaussians and width * height <= 65,536 pixels (larger
 * inputs are rejected with QR_ERR_INVALID_ARG before anything is launched),
 * and at most 524,288 tile-Gaussian intersections (an overflow is reported
 * by qr_frame_status on *frame_out, which describes the static workspace
 * until the next call; frame_out may be NULL).
 * The first call on each device looks up the array's device address
 * (cudaGetSymbolAddress, with that device current) and keeps it for the rest
 * of the process; make that first call before any stream capture, and do not
 * reset the device (cudaDeviceReset) after it, which would leave the kept
 * address stale.  All calls share the one array: calls that overlap on the
 * GPU race.  A call allocates nothing: no cudaMalloc, no cudaFree, no
 * allocating library routine. */
qr_status qr_render_noalloc(const float *mean, const float *log_scale, const float *quat,
                            const float *opacity, int64_t n, const qr_camera *camera,
                            const qr_params *params, const void *feat, const float *feat_scale,
                            qr_dtype dtype, int32_t C, int32_t *ids, float *weights,
                            uint8_t *counts, float *out, qr_frame *frame_out, qr_stream stream);

/* ---------------------------------------------------------------- instrumentation */

/* Number of kernels this library has launched since it was loaded. */
uint64_t qr_launch_count(void);

/* Test hook for the device-side error path.  The relevance kernels
 * (qr_relevance's TMA kernel, qr_blend_relevance) bound each of their waits
 * on a producer, the tensor cores or the epilogue to a number of polls
 * (2^26 by default, seconds); when one runs out the CTA stops every role,
 * waits (with the default bound) for its own copies and MMAs in flight,
 * frees its tensor memory and writes QR_ERR_DEVICE_TIMEOUT to the call's
 * status word.  qr_set_wait_limit(polls) sets that bound for the launches
 * that follow (0 restores the default), so a test can make a wait run out
 * without anything hanging.  Not for production use; not thread-safe. */
void qr_set_wait_limit(uint32_t polls);

/* Tuning: the blend of 512-D rows (any dtype) with K <= 8 splits each
 * feature row into `chunks` channel slices taken by different warps (1, 2 or
 * 4; 0 restores the built-in choice, one slice; wider rows always use the
 * built-in choice: at most 16 accumulators per pixel and lane).  More chunks
 * mean fewer registers per thread and more warps per SM.  The sums and their
 * order per channel do not change, so results are bit-identical for every
 * setting.  Applies to qr_blend and qr_render launched afterwards; returns
 * QR_ERR_INVALID_ARG for other values.  Not thread-safe. */
qr_status qr_set_blend_chunks(int32_t chunks);

#ifdef __cplusplus
}
#endif

#endif /* QRENDER_H */
