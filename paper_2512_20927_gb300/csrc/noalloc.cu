// qr_render_noalloc: the Q-Render forward of qr_render for callers that cannot
// allocate device memory.
//
// Some callers of a renderer may not call cudaMalloc (or any allocating
// routine) at all: a plug-in whose host application owns every byte of device
// memory through its own pool, a hard real-time loop in which an allocation
// may block or fail, or code that sets everything up before a CUDA graph is
// recorded.  They still pass their inputs and outputs; the scratch that
// qr_render takes from a caller-sized workspace lives here instead, in one
// static device array that every GPU loading the library holds until the
// process exits.
//
// Limits: at most kMaxGaussians Gaussians, kMaxPixels pixels and kMaxIsect
// tile-Gaussian intersections (a larger frame reports QR_ERR_CAPACITY through
// qr_frame_status on the returned frame).  All calls share the array: calls
// that overlap on the GPU (different streams, or different host threads
// without ordering) race and corrupt each other's results.  Each call starts
// by clearing the status counters and tile ranges it depends on; everything
// else it reads it has written earlier in the same call.
#include <mutex>

#include "qr_internal.cuh"

namespace {

constexpr int64_t kMaxGaussians = 65536;
constexpr int64_t kMaxPixels = 65536;
constexpr int64_t kMaxIsect = 524288;
constexpr size_t kScratchBytes = size_t(16) << 20;   // 16 MiB

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

std::mutex g_mu;
constexpr int kMaxDevices = 256;
void *g_scratch_ptr[kMaxDevices] = {};

// Device address of the static array on the current device, resolved once per
// device with that device current.  In host code the array's name is only a
// stand-in: its device address must come from cudaGetSymbolAddress.
qr_status scratch_for_current_device(void **out) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return QR_ERR_CUDA;
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_ptr[dev]) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || p == nullptr) return QR_ERR_CUDA;
        g_scratch_ptr[dev] = p;
    }
    *out = g_scratch_ptr[dev];
    return QR_OK;
}

}  // namespace

extern "C" qr_status qr_render_noalloc(const float *mean, const float *log_scale,
                                       const float *quat, const float *opacity, int64_t n,
                                       const qr_camera *camera, const qr_params *params,
                                       const void *feat, const float *feat_scale, qr_dtype dtype,
                                       int32_t C, int32_t *ids, float *weights, uint8_t *counts,
                                       float *out, qr_frame *frame_out, qr_stream stream) {
    if (!camera || !params) return QR_ERR_INVALID_ARG;
    if (n < 0 || n > kMaxGaussians) return QR_ERR_INVALID_ARG;
    if (camera->width < 1 || camera->height < 1 ||
        int64_t(camera->width) * int64_t(camera->height) > kMaxPixels)
        return QR_ERR_INVALID_ARG;
    const size_t need = qr_workspace_bytes(n, camera->width, camera->height, params, kMaxIsect);
    if (need == 0 || need > kScratchBytes) return QR_ERR_INVALID_ARG;
    void *ws = nullptr;
    qr_status st = scratch_for_current_device(&ws);
    if (st != QR_OK) return st;
    qr_frame f;
    st = qr_frame_init(&f, n, camera, params, kMaxIsect, ws, kScratchBytes);
    if (st != QR_OK) return st;
    st = qr_render(&f, mean, log_scale, quat, opacity, feat, feat_scale, dtype, C, ids, weights,
                   counts, out, stream);
    if (st == QR_OK && frame_out) *frame_out = f;
    return st;
}
