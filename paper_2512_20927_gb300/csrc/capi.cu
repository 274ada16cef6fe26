// C ABI of libqrender: argument checks, workspace layout and the composed
// calls.  Every entry point validates on the host and launches nothing when
// it returns an error.
#include <atomic>
#include <cmath>
#include <cstring>
#include <vector>

#include "qr_internal.cuh"

namespace qr {

static std::atomic<uint64_t> g_launches{0};
void count_launch(int n) { g_launches.fetch_add(uint64_t(n), std::memory_order_relaxed); }

bool blend_supported(qr_dtype dt, int C);
bool dense_supported(qr_dtype dt, int C);
cudaError_t launch_blend_tiled(const void *feat, const float *scale, qr_dtype dt, int C,
                               int64_t n_gauss, const int32_t *ids, const float *w,
                               const uint8_t *cnt, int64_t P, int K, int W, int H, float *out,
                               cudaStream_t s);

namespace {

constexpr size_t kAlign = 256;
inline size_t align_up(size_t x, size_t a = kAlign) { return (x + a - 1) / a * a; }
inline bool aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

bool params_ok(const qr_params *p) {
    if (!p) return false;
    if (p->K < 1 || p->K > kKMax) return false;
    if (!(p->alpha_min > 0.f && p->alpha_min < p->alpha_max && p->alpha_max < 1.f)) return false;
    if (!(p->T_min >= 0.f && p->T_min < 1.f)) return false;
    if (!(p->dilation >= 0.f)) return false;
    if (p->tile_w * p->tile_h != 256) return false;
    if (p->tile_w != 8 && p->tile_w != 16 && p->tile_w != 32) return false;
    return true;
}

bool dims_ok(int64_t n, int W, int H, int64_t cap) {
    if (n < 0 || n > int64_t(0x7FFFFFFF)) return false;
    if (W < 1 || H < 1 || int64_t(W) * H > int64_t(0x7FFFFFFF)) return false;
    if (cap < 0 || cap > int64_t(0xFFFFFFFEu)) return false;
    return true;
}

// Compute slot offsets; returns total bytes (0 on invalid input).
size_t layout(int64_t n, int W, int H, const qr_params *p, int64_t cap, size_t *off) {
    if (!params_ok(p) || !dims_ok(n, W, H, cap)) return 0;
    const int64_t tx = (W + p->tile_w - 1) / p->tile_w, ty = (H + p->tile_h - 1) / p->tile_h;
    if (tx > 65535 || ty > 65535) return 0;
    const size_t N = size_t(n), X = size_t(cap), tiles = size_t(tx * ty);
    size_t sizes[S_END];
    const size_t nblk = (N + kProjectThreads - 1) / kProjectThreads + 1;
    sizes[S_COUNTERS] = CNT_WORDS * 4;
    sizes[S_REC_M] = N * 16;
    sizes[S_REC_C] = N * 16;
    sizes[S_REC_A] = N * 4;
    sizes[S_REC_H] = N * 4;
    sizes[S_RECT] = N * 8;
    sizes[S_TCOUNT] = N * 4;
    sizes[S_GKEY] = N * 4;
    sizes[S_VISCNT] = nblk * 4;
    sizes[S_BSUM] = nblk * 4;
    sizes[S_KID] = N * 4;
    sizes[S_OFF] = N * 4;
    sizes[S_TCNT] = tiles * 4;
    sizes[S_RANGES] = tiles * 8;
    sizes[S_KEYS64] = X * 8;
    sizes[S_SCRATCH64] = X * 8;
    sizes[S_IGID] = X * 4;
    sizes[S_DIFF] = size_t(tx + 1) * size_t(ty + 1) * 4 * kDiffCopies;
    sizes[S_CHUNK] = (X / kEmitChunk + 2) * 4;
    size_t o = 0;
    for (int s = 0; s < S_END; ++s) {
        if (off) off[s] = o;
        o = align_up(o + (sizes[s] ? sizes[s] : 1));
    }
    return o;
}

qr_status from_cuda(cudaError_t e) { return e == cudaSuccess ? QR_OK : QR_ERR_CUDA; }

// (L, 1/n) of a loss over no pixels: L = 0, n floored at 1.
const float kEmptyLoss[2] = {0.0f, 1.0f};

bool frame_ok(const qr_frame *f) {
    return f && f->ws && params_ok(&f->params) && dims_ok(f->n, f->camera.width, f->camera.height, f->max_isect);
}

}  // namespace
}  // namespace qr

using namespace qr;

extern "C" {

int32_t qr_abi_version(void) { return 1; }

const char *qr_status_string(qr_status s) {
    switch (s) {
        case QR_OK: return "ok";
        case QR_ERR_INVALID_ARG: return "invalid argument";
        case QR_ERR_ALIGNMENT: return "misaligned pointer or row";
        case QR_ERR_CAPACITY: return "intersection capacity exceeded";
        case QR_ERR_CUDA: return "CUDA runtime error";
        case QR_ERR_DEVICE_TIMEOUT: return "device-side wait timed out";
        case QR_ERR_NOT_SUPPORTED: return "not supported";
    }
    return "unknown status";
}

void qr_default_params(qr_params *p) {
    if (!p) return;
    p->K = 8;
    p->alpha_min = 1.0f / 255.0f;
    p->alpha_max = 0.99f;
    p->T_min = 1e-4f;
    p->dilation = 0.3f;
    p->tile_w = 16;
    p->tile_h = 16;
}

size_t qr_workspace_bytes(int64_t n, int32_t width, int32_t height, const qr_params *params,
                          int64_t max_isect) {
    return layout(n, width, height, params, max_isect, nullptr);
}

qr_status qr_frame_init(qr_frame *frame, int64_t n, const qr_camera *camera,
                        const qr_params *params, int64_t max_isect, void *ws, size_t ws_bytes) {
    if (!frame || !camera || !params || !ws) return QR_ERR_INVALID_ARG;
    if ((reinterpret_cast<uintptr_t>(ws) & (kAlign - 1)) != 0) return QR_ERR_ALIGNMENT;
    for (int i = 0; i < 9; ++i)
        if (!std::isfinite(camera->R[i])) return QR_ERR_INVALID_ARG;
    for (int i = 0; i < 3; ++i)
        if (!std::isfinite(camera->t[i])) return QR_ERR_INVALID_ARG;
    if (!(camera->fx > 0.f && camera->fy > 0.f && std::isfinite(camera->fx) && std::isfinite(camera->fy) &&
          std::isfinite(camera->cx) && std::isfinite(camera->cy) && camera->near_plane > 0.f &&
          std::isfinite(camera->near_plane)))
        return QR_ERR_INVALID_ARG;
    qr_frame f;
    std::memset(&f, 0, sizeof(f));
    const size_t need = layout(n, camera->width, camera->height, params, max_isect, f.off);
    if (need == 0 || ws_bytes < need) return QR_ERR_INVALID_ARG;
    f.n = n;
    f.max_isect = max_isect;
    f.camera = *camera;
    f.params = *params;
    f.tiles_x = (camera->width + params->tile_w - 1) / params->tile_w;
    f.tiles_y = (camera->height + params->tile_h - 1) / params->tile_h;
    f.sort_blocks = 0;   // reserved
    f.isect_buf = 0;
    f.ws = ws;
    f.ws_bytes = ws_bytes;
    *frame = f;
    return QR_OK;
}

qr_status qr_frame_view_get(const qr_frame *frame, qr_frame_view *view) {
    if (!frame_ok(frame) || !view) return QR_ERR_INVALID_ARG;
    const qr_frame &f = *frame;
    view->mean2d_hi_lo = slot<float>(f, S_REC_M);
    view->axes = slot<float>(f, S_REC_C);
    view->opacity = slot<float>(f, S_REC_A);
    view->depth_key = slot<uint32_t>(f, S_GKEY);
    view->tile_count = slot<uint32_t>(f, S_TCOUNT);
    view->kept_gid = slot<uint32_t>(f, S_KID);
    view->kept_offset = slot<uint32_t>(f, S_OFF);
    view->isect_gid = slot<uint32_t>(f, S_IGID);
    view->tile_range = slot<uint32_t>(f, S_RANGES);
    view->counters = slot<uint32_t>(f, S_COUNTERS);
    return QR_OK;
}

qr_status qr_frame_status(const qr_frame *frame, qr_stream stream, int64_t *n_isect) {
    if (!frame_ok(frame)) return QR_ERR_INVALID_ARG;
    cudaError_t e = cudaStreamSynchronize(reinterpret_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return QR_ERR_CUDA;
    uint32_t c[CNT_WORDS];
    e = cudaMemcpy(c, slot<uint32_t>(*frame, S_COUNTERS), sizeof(c), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return QR_ERR_CUDA;
    if (n_isect) *n_isect = int64_t(c[CNT_ISECT]);
    return c[CNT_STATUS] == 0 ? QR_OK : qr_status(c[CNT_STATUS]);
}

qr_status qr_project(qr_frame *frame, const float *mean, const float *log_scale,
                     const float *quat, const float *opacity, qr_stream stream) {
    if (!frame_ok(frame)) return QR_ERR_INVALID_ARG;
    if (frame->n > 0 && (!mean || !log_scale || !quat || !opacity)) return QR_ERR_INVALID_ARG;
    return from_cuda(launch_project(*frame, mean, log_scale, quat, opacity,
                                    reinterpret_cast<cudaStream_t>(stream)));
}

qr_status qr_sort(qr_frame *frame, qr_stream stream) {
    if (!frame_ok(frame)) return QR_ERR_INVALID_ARG;
    return from_cuda(launch_sort(*frame, reinterpret_cast<cudaStream_t>(stream)));
}

qr_status qr_select(const qr_frame *frame, int32_t *ids, float *weights, uint8_t *counts,
                    qr_stream stream) {
    if (!frame_ok(frame) || !ids || !weights || !counts) return QR_ERR_INVALID_ARG;
    return from_cuda(launch_select(*frame, ids, weights, counts, false,
                                   reinterpret_cast<cudaStream_t>(stream)));
}

qr_status qr_select_rule(const qr_frame *frame, qr_rule rule, int32_t *ids, float *weights,
                         uint8_t *counts, float *tau, qr_stream stream) {
    if (!frame_ok(frame) || !ids || !weights || !counts) return QR_ERR_INVALID_ARG;
    if (rule != QR_RULE_QUANTILE && rule != QR_RULE_TOPK && rule != QR_RULE_STRATIFIED &&
        rule != QR_RULE_RIEMANN)
        return QR_ERR_INVALID_ARG;
    const cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    if (rule == QR_RULE_QUANTILE || rule == QR_RULE_RIEMANN)
        return from_cuda(launch_select(*frame, ids, weights, counts, rule == QR_RULE_RIEMANN, s));
    return from_cuda(launch_select_rule(*frame, int(rule), ids, weights, counts,
                                        rule == QR_RULE_STRATIFIED ? tau : nullptr, s));
}

static qr_status check_feat(const void *feat, const float *feat_scale, qr_dtype dtype, int32_t C) {
    if (!feat || C <= 0) return QR_ERR_INVALID_ARG;
    if (dtype != QR_F32 && dtype != QR_BF16 && dtype != QR_FP8E4M3) return QR_ERR_INVALID_ARG;
    if (dtype == QR_FP8E4M3 && !feat_scale) return QR_ERR_INVALID_ARG;
    const int esz = dtype == QR_F32 ? 4 : dtype == QR_BF16 ? 2 : 1;
    if (!aligned16(feat) || (size_t(C) * esz) % 16 != 0) return QR_ERR_ALIGNMENT;
    return QR_OK;
}

qr_status qr_blend(const void *feat, const float *feat_scale, qr_dtype dtype, int32_t C,
                   int64_t n_gauss, const int32_t *ids, const float *weights,
                   const uint8_t *counts, int64_t P, int32_t K, int32_t width, float *out,
                   qr_stream stream) {
    qr_status st = check_feat(feat, feat_scale, dtype, C);
    if (st != QR_OK) return st;
    if (!ids || !weights || !counts || !out || P < 0 || K < 1 || K > kKMax || n_gauss < 1 ||
        width < 0 || (width > 0 && P % width != 0))
        return QR_ERR_INVALID_ARG;
    if (!aligned16(out)) return QR_ERR_ALIGNMENT;
    if (!blend_supported(dtype, C)) return QR_ERR_NOT_SUPPORTED;
    if (P == 0) return QR_OK;
    const int H = width > 0 ? int(P / width) : 0;
    return from_cuda(launch_blend_tiled(feat, feat_scale, dtype, C, n_gauss, ids, weights, counts,
                                        P, K, width, H, out, reinterpret_cast<cudaStream_t>(stream)));
}

qr_status qr_dense(const qr_frame *frame, const void *feat, const float *feat_scale,
                   qr_dtype dtype, int32_t C, float *out, float *T_final, qr_stream stream) {
    if (!frame_ok(frame) || !out) return QR_ERR_INVALID_ARG;
    qr_status st = check_feat(feat, feat_scale, dtype, C);
    if (st != QR_OK) return st;
    if (!aligned16(out)) return QR_ERR_ALIGNMENT;
    if (!dense_supported(dtype, C)) return QR_ERR_NOT_SUPPORTED;
    return from_cuda(launch_dense(*frame, feat, feat_scale, dtype, C, out, T_final,
                                  reinterpret_cast<cudaStream_t>(stream)));
}

qr_status qr_dense_work(const qr_frame *frame, const void *feat, const float *feat_scale,
                        qr_dtype dtype, int32_t C, float *out, float *T_final, uint64_t *counts,
                        qr_stream stream) {
    if (!frame_ok(frame) || !out || !counts) return QR_ERR_INVALID_ARG;
    qr_status st = check_feat(feat, feat_scale, dtype, C);
    if (st != QR_OK) return st;
    if (!aligned16(out)) return QR_ERR_ALIGNMENT;
    if (!dense_supported(dtype, C)) return QR_ERR_NOT_SUPPORTED;
    const cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    cudaError_t e = cudaMemsetAsync(counts, 0, 2 * sizeof(uint64_t), s);
    if (e != cudaSuccess) return QR_ERR_CUDA;
    return from_cuda(launch_dense(*frame, feat, feat_scale, dtype, C, out, T_final, s,
                                  reinterpret_cast<unsigned long long *>(counts)));
}

qr_status qr_render(qr_frame *frame, const float *mean, const float *log_scale,
                    const float *quat, const float *opacity, const void *feat,
                    const float *feat_scale, qr_dtype dtype, int32_t C, int32_t *ids,
                    float *weights, uint8_t *counts, float *out, qr_stream stream) {
    if (!frame_ok(frame) || !ids || !weights || !counts || !out) return QR_ERR_INVALID_ARG;
    qr_status st = check_feat(feat, feat_scale, dtype, C);
    if (st != QR_OK) return st;
    if (!aligned16(out)) return QR_ERR_ALIGNMENT;
    if (!blend_supported(dtype, C)) return QR_ERR_NOT_SUPPORTED;
    if (frame->n > 0 && (!mean || !log_scale || !quat || !opacity)) return QR_ERR_INVALID_ARG;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    cudaError_t e = launch_project(*frame, mean, log_scale, quat, opacity, s);
    if (e == cudaSuccess) e = launch_sort(*frame, s);
    if (e == cudaSuccess) e = launch_select(*frame, ids, weights, counts, false, s);
    if (e == cudaSuccess)
        e = launch_blend_tiled(feat, feat_scale, dtype, C, frame->n > 0 ? frame->n : 1, ids, weights,
                               counts, num_pixels(*frame), frame->params.K, 0, 0, out, s);
    return from_cuda(e);
}

static size_t esize(qr_dtype d) { return d == QR_F32 ? 4 : d == QR_BF16 ? 2 : 1; }

qr_status qr_render_host_bytes(int64_t n, int32_t width, int32_t height, int32_t K, int32_t C,
                               qr_dtype dtype, size_t *dev_inputs_bytes,
                               size_t *dev_outputs_bytes) {
    if (n < 0 || width < 1 || height < 1 || K < 1 || K > kKMax || C < 1) return QR_ERR_INVALID_ARG;
    const size_t N = size_t(n), P = size_t(width) * size_t(height);
    if (dev_inputs_bytes)
        *dev_inputs_bytes = align_up(N * 11 * 4) + align_up(N * size_t(C) * esize(dtype)) + align_up(N * 4);
    if (dev_outputs_bytes)
        *dev_outputs_bytes = align_up(P * K * 4) * 2 + align_up(P) + align_up(P * size_t(C) * 4);
    return QR_OK;
}

qr_status qr_render_host(qr_frame *frame, const float *mean_host, const float *log_scale_host,
                         const float *quat_host, const float *opacity_host,
                         const void *feat_host, const float *feat_scale_host, qr_dtype dtype,
                         int32_t C, void *dev_inputs, void *dev_outputs, float *out_host,
                         qr_stream stream) {
    if (!frame_ok(frame) || !dev_inputs || !dev_outputs || !out_host || !feat_host) return QR_ERR_INVALID_ARG;
    if (frame->n > 0 && (!mean_host || !log_scale_host || !quat_host || !opacity_host))
        return QR_ERR_INVALID_ARG;
    if (dtype == QR_FP8E4M3 && !feat_scale_host) return QR_ERR_INVALID_ARG;
    if ((reinterpret_cast<uintptr_t>(dev_inputs) & (kAlign - 1)) ||
        (reinterpret_cast<uintptr_t>(dev_outputs) & (kAlign - 1)))
        return QR_ERR_ALIGNMENT;
    const size_t N = size_t(frame->n), P = size_t(num_pixels(*frame)), K = size_t(frame->params.K);
    char *in = static_cast<char *>(dev_inputs);
    float *d_mean = reinterpret_cast<float *>(in);
    float *d_ls = d_mean + 3 * N;
    float *d_q = d_ls + 3 * N;
    float *d_op = d_q + 4 * N;
    void *d_feat = in + align_up(N * 11 * 4);
    float *d_scale = reinterpret_cast<float *>(in + align_up(N * 11 * 4) + align_up(N * size_t(C) * esize(dtype)));
    char *outb = static_cast<char *>(dev_outputs);
    int32_t *d_ids = reinterpret_cast<int32_t *>(outb);
    float *d_w = reinterpret_cast<float *>(outb + align_up(P * K * 4));
    uint8_t *d_cnt = reinterpret_cast<uint8_t *>(outb + 2 * align_up(P * K * 4));
    float *d_map = reinterpret_cast<float *>(outb + 2 * align_up(P * K * 4) + align_up(P));
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    cudaError_t e = cudaSuccess;
    if (N) {
        e = cudaMemcpyAsync(d_mean, mean_host, N * 12, cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(d_ls, log_scale_host, N * 12, cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(d_q, quat_host, N * 16, cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(d_op, opacity_host, N * 4, cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(d_feat, feat_host, N * size_t(C) * esize(dtype), cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess && dtype == QR_FP8E4M3)
            e = cudaMemcpyAsync(d_scale, feat_scale_host, N * 4, cudaMemcpyHostToDevice, s);
        if (e != cudaSuccess) return QR_ERR_CUDA;
    }
    qr_status st = qr_render(frame, d_mean, d_ls, d_q, d_op, d_feat,
                             dtype == QR_FP8E4M3 ? d_scale : nullptr, dtype, C, d_ids, d_w, d_cnt,
                             d_map, stream);
    if (st != QR_OK) return st;
    e = cudaMemcpyAsync(out_host, d_map, P * size_t(C) * 4, cudaMemcpyDeviceToHost, s);
    return from_cuda(e);
}

size_t qr_backward_workspace_bytes(const qr_frame *frame, int32_t C) {
    if (!frame_ok(frame) || C < 4 || C % 4) return 0;
    return backward_workspace_bytes(*frame, C);
}

qr_status qr_backward(const qr_frame *frame, const void *feat, const float *feat_scale,
                      qr_dtype dtype, int32_t C, const int32_t *ids, const float *weights,
                      const uint8_t *counts, const float *grad_out, float *grad_feat,
                      float *grad_opacity, float *grad_conic, void *ws, size_t ws_bytes,
                      qr_stream stream) {
    if (!frame_ok(frame) || !ids || !weights || !counts || !grad_out || !grad_feat || !ws)
        return QR_ERR_INVALID_ARG;
    qr_status st = check_feat(feat, feat_scale, dtype, C);
    if (st != QR_OK) return st;
    if (!aligned16(grad_out) || !aligned16(grad_feat) ||
        (reinterpret_cast<uintptr_t>(ws) & (kAlign - 1)))
        return QR_ERR_ALIGNMENT;
    if (ws_bytes < backward_workspace_bytes(*frame, C)) return QR_ERR_INVALID_ARG;
    if (frame->n == 0) return QR_OK;
    return from_cuda(launch_backward(*frame, feat, feat_scale, dtype, C, ids, weights, counts,
                                     grad_out, grad_feat, grad_opacity, grad_conic, ws,
                                     reinterpret_cast<cudaStream_t>(stream)));
}

size_t qr_cosine_backward_workspace_bytes(const qr_frame *frame, int32_t C) {
    if (!frame_ok(frame) || C < 4 || C % 4) return 0;
    return backward_cos_workspace_bytes(*frame, C);
}

qr_status qr_cosine_backward(const qr_frame *frame, const void *feat, const float *feat_scale,
                             qr_dtype dtype, int32_t C, const int32_t *ids, const float *weights,
                             const uint8_t *counts, const float *feature_map, const float *target,
                             const uint8_t *mask, float *loss_out, float *grad_map,
                             float *grad_feat, float *grad_opacity, float *grad_conic, void *ws,
                             size_t ws_bytes, qr_stream stream) {
    if (!frame_ok(frame) || !ids || !weights || !counts || !feature_map || !target || !mask ||
        !loss_out || !grad_map || !grad_feat || !ws)
        return QR_ERR_INVALID_ARG;
    qr_status st = check_feat(feat, feat_scale, dtype, C);
    if (st != QR_OK) return st;
    if (!aligned16(feature_map) || !aligned16(target) || !aligned16(grad_map) ||
        !aligned16(grad_feat) || (reinterpret_cast<uintptr_t>(ws) & (kAlign - 1)))
        return QR_ERR_ALIGNMENT;
    if (ws_bytes < backward_cos_workspace_bytes(*frame, C)) return QR_ERR_INVALID_ARG;
    const int64_t P = num_pixels(*frame);
    const cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    if (P == 0)
        return from_cuda(cudaMemcpyAsync(loss_out, kEmptyLoss, sizeof(kEmptyLoss),
                                         cudaMemcpyHostToDevice, s));
    CosLossArgs loss;
    loss.F = feature_map;
    loss.tgt = target;
    loss.mask = mask;
    loss.term = reinterpret_cast<float *>(static_cast<char *>(ws) + backward_workspace_bytes(*frame, C));
    loss.out2 = loss_out;
    loss.grad_map = grad_map;
    if (frame->n == 0)   // nothing to differentiate: the loss alone
        return from_cuda(launch_cosine_loss(feature_map, target, mask, P, C, loss.term, loss_out,
                                            grad_map, s));
    return from_cuda(launch_backward_cos(*frame, feat, feat_scale, dtype, C, ids, weights, counts,
                                         loss, grad_feat, grad_opacity, grad_conic, ws, s));
}

qr_status qr_cosine_loss(const float *feature_map, const float *target, const uint8_t *counts,
                         int64_t P, int32_t C, float *loss_out, float *grad, float *scratch,
                         qr_stream stream) {
    if (!feature_map || !target || !counts || !loss_out || !grad || !scratch || P < 0 || C < 1)
        return QR_ERR_INVALID_ARG;
    if (P == 0)
        return from_cuda(cudaMemcpyAsync(loss_out, kEmptyLoss, sizeof(kEmptyLoss),
                                         cudaMemcpyHostToDevice,
                                         reinterpret_cast<cudaStream_t>(stream)));
    return from_cuda(launch_cosine_loss(feature_map, target, counts, P, C, scratch, loss_out, grad,
                                        reinterpret_cast<cudaStream_t>(stream)));
}

size_t qr_contrastive_workspace_bytes(int64_t P, int32_t M, int32_t C) {
    if (P < 0 || !contrastive_supported(M, C)) return 0;
    return contrastive_workspace_bytes(P, M, C);
}

qr_status qr_contrastive_loss(const float *feature_map, const float *targets, int32_t M,
                              int32_t C, const int32_t *mask_id, int64_t P, float *loss_out,
                              float *grad, void *ws, size_t ws_bytes, qr_stream stream) {
    if (!feature_map || !targets || !mask_id || !loss_out || !grad || !ws || P < 0)
        return QR_ERR_INVALID_ARG;
    if (!contrastive_supported(M, C)) return QR_ERR_NOT_SUPPORTED;
    if (!aligned16(feature_map) || !aligned16(targets) || !aligned16(grad) ||
        (reinterpret_cast<uintptr_t>(ws) & (kAlign - 1)))
        return QR_ERR_ALIGNMENT;
    if (ws_bytes < contrastive_workspace_bytes(P, M, C)) return QR_ERR_INVALID_ARG;
    const cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    if (P == 0)
        return from_cuda(cudaMemcpyAsync(loss_out, kEmptyLoss, sizeof(kEmptyLoss),
                                         cudaMemcpyHostToDevice, s));
    return from_cuda(launch_contrastive_loss(feature_map, targets, M, C, mask_id, P, loss_out,
                                             grad, ws, s));
}

size_t qr_contrastive_backward_workspace_bytes(const qr_frame *frame, int32_t M, int32_t C) {
    if (!frame_ok(frame) || C < 4 || C % 4 || !contrastive_supported(M, C)) return 0;
    return align_up(backward_workspace_bytes(*frame, C)) +
           contrastive_workspace_bytes(num_pixels(*frame), M, C);
}

qr_status qr_contrastive_backward(const qr_frame *frame, const void *feat, const float *feat_scale,
                                  qr_dtype dtype, int32_t C, const int32_t *ids,
                                  const float *weights, const uint8_t *counts,
                                  const float *feature_map, const float *targets, int32_t M,
                                  const int32_t *mask_id, float *loss_out, float *grad_map,
                                  float *grad_feat, float *grad_opacity, float *grad_conic,
                                  void *ws, size_t ws_bytes, qr_stream stream) {
    if (!frame_ok(frame) || !ids || !weights || !counts || !feature_map || !targets || !mask_id ||
        !loss_out || !grad_map || !grad_feat || !ws)
        return QR_ERR_INVALID_ARG;
    qr_status st = check_feat(feat, feat_scale, dtype, C);
    if (st != QR_OK) return st;
    if (!contrastive_supported(M, C)) return QR_ERR_NOT_SUPPORTED;
    if (!aligned16(feature_map) || !aligned16(targets) || !aligned16(grad_map) ||
        !aligned16(grad_feat) || (reinterpret_cast<uintptr_t>(ws) & (kAlign - 1)))
        return QR_ERR_ALIGNMENT;
    const size_t bw = align_up(backward_workspace_bytes(*frame, C));
    const int64_t P = num_pixels(*frame);
    if (ws_bytes < bw + contrastive_workspace_bytes(P, M, C)) return QR_ERR_INVALID_ARG;
    const cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    cudaError_t e = launch_contrastive_loss(feature_map, targets, M, C, mask_id, P, loss_out,
                                            grad_map, static_cast<char *>(ws) + bw, s);
    if (e != cudaSuccess) return QR_ERR_CUDA;
    if (frame->n == 0) return QR_OK;
    return from_cuda(launch_backward(*frame, feat, feat_scale, dtype, C, ids, weights, counts,
                                     grad_map, grad_feat, grad_opacity, grad_conic, ws, s));
}

qr_status qr_blend_relevance(const void *feat, const float *feat_scale, qr_dtype dtype, int32_t C,
                             int64_t n_gauss, const int32_t *ids, const float *weights,
                             const uint8_t *counts, int64_t P, int32_t K, int32_t width,
                             const uint16_t *queries_bf16, int32_t Q, float *out, int32_t *status,
                             qr_stream stream) {
    qr_status st = check_feat(feat, feat_scale, dtype, C);
    if (st != QR_OK) return st;
    if (!ids || !weights || !counts || !queries_bf16 || !out || !status || P < 0 || n_gauss < 1 ||
        width < 0 || (width > 0 && P % width != 0))
        return QR_ERR_INVALID_ARG;
    if (!blend_relevance_supported(dtype, Q, C, K)) return QR_ERR_NOT_SUPPORTED;
    if (!aligned16(queries_bf16) || !aligned16(out)) return QR_ERR_ALIGNMENT;
    if (P == 0) return QR_OK;
    const int H = width > 0 ? int(P / width) : 0;
    return from_cuda(launch_blend_relevance(feat, feat_scale, dtype, C, n_gauss, ids, weights,
                                            counts, P, K, width, H, queries_bf16, Q, out, status,
                                            reinterpret_cast<cudaStream_t>(stream)));
}

qr_status qr_relevance(const float *feature_map, const uint16_t *queries_bf16, int32_t Q, int32_t C,
                       int64_t P, float *out, int32_t *status, qr_stream stream) {
    if (!feature_map || !queries_bf16 || !out || !status || P < 0) return QR_ERR_INVALID_ARG;
    if (!relevance_supported(Q, C)) return QR_ERR_NOT_SUPPORTED;
    if (!aligned16(feature_map) || !aligned16(queries_bf16) || !aligned16(out)) return QR_ERR_ALIGNMENT;
    if (P == 0) return QR_OK;
    return from_cuda(launch_relevance(feature_map, queries_bf16, Q, P, C, out, status,
                                      reinterpret_cast<cudaStream_t>(stream)));
}

size_t qr_batch_workspace_bytes(int32_t n_views) {
    return n_views < 1 ? 0 : batch_desc_bytes(n_views);
}

qr_status qr_batch_prepare(const qr_view *views, int32_t n_views, void *ws, size_t ws_bytes,
                           uint32_t *total_tiles, qr_stream stream) {
    if (!views || n_views < 1 || !ws || !total_tiles) return QR_ERR_INVALID_ARG;
    if ((reinterpret_cast<uintptr_t>(ws) & (kAlign - 1)) != 0) return QR_ERR_ALIGNMENT;
    if (ws_bytes < batch_desc_bytes(n_views)) return QR_ERR_INVALID_ARG;
    uint64_t tiles = 0;
    for (int i = 0; i < n_views; ++i) {
        const qr_view &v = views[i];
        if (!frame_ok(v.frame) || !v.feat || !v.ids || !v.weights || !v.counts || !v.out)
            return QR_ERR_INVALID_ARG;
        if (v.frame->params.K != views[0].frame->params.K) return QR_ERR_INVALID_ARG;
        if (!aligned16(v.feat) || !aligned16(v.out)) return QR_ERR_ALIGNMENT;
        tiles += uint64_t(num_tiles(*v.frame));
    }
    if (tiles > 0xFFFFFFF0ull) return QR_ERR_INVALID_ARG;
    std::vector<unsigned char> host(batch_view_size() * size_t(n_views));
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    cudaError_t e = prepare_batch(views, n_views, ws, total_tiles, s,
                                  reinterpret_cast<BatchView *>(host.data()));
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    return from_cuda(e);
}

qr_status qr_render_batch(const void *ws, int32_t n_views, uint32_t total_tiles, qr_dtype dtype,
                          int32_t C, int32_t K, int32_t group, int32_t chunks,
                          int32_t blend_warps, int32_t ctas_per_sm, qr_stream stream) {
    if (!ws || n_views < 1 || K < 1 || K > kKMax || group < 0 || group > 4 || ctas_per_sm < 0)
        return QR_ERR_INVALID_ARG;
    if (dtype != QR_F32 && dtype != QR_BF16 && dtype != QR_FP8E4M3) return QR_ERR_INVALID_ARG;
    if (!batch_supported(dtype, C)) return QR_ERR_NOT_SUPPORTED;
    if (chunks != 0 && chunks != 1 && chunks != 2 && chunks != 4) return QR_ERR_INVALID_ARG;
    if (blend_warps != 0 && blend_warps != 4 && blend_warps != 8) return QR_ERR_INVALID_ARG;
    if (!batch_chunks_ok(C, chunks)) return QR_ERR_INVALID_ARG;
    if (total_tiles == 0) return QR_OK;
    return from_cuda(launch_batch(ws, n_views, total_tiles, dtype, C, K, group, chunks, blend_warps,
                                  ctas_per_sm, reinterpret_cast<cudaStream_t>(stream)));
}

uint64_t qr_launch_count(void) { return g_launches.load(std::memory_order_relaxed); }

void qr_set_wait_limit(uint32_t polls) { set_wait_limit(polls); }

qr_status qr_set_blend_chunks(int32_t chunks) {
    return set_blend_chunks(chunks) ? QR_OK : QR_ERR_INVALID_ARG;
}

}  // extern "C"
