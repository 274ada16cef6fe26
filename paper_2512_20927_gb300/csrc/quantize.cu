// Storage formats of the feature table (not in the paper): BF16, and FP8 E4M3
// with one FP32 scale per Gaussian.  The blend and dense kernels decode both
// in registers and accumulate in FP32.
//
// BF16: round to nearest, ties to even (__float2bfloat16_rn).
// FP8:  scale_i = max_c |f_ic| / 448 (1 for an all-zero row), computed in FP32;
//       code_ic = E4M3(f_ic / scale_i) with the division rounded to nearest and
//       the conversion rounding to nearest even and saturating to +-448.
// One warp per row for FP8 (max by shuffles, then 16-byte code stores).
#include <cuda_bf16.h>
#include <cuda_fp8.h>

#include "qr_internal.cuh"

namespace qr {
namespace {

__global__ void __launch_bounds__(256)
bf16_kernel(const float *__restrict__ in, int64_t count, uint16_t *__restrict__ out) {
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < count; i += stride) {
        const __nv_bfloat16 b = __float2bfloat16_rn(in[i]);
        out[i] = *reinterpret_cast<const uint16_t *>(&b);
    }
}

__global__ void __launch_bounds__(256)
fp8_rows_kernel(const float *__restrict__ in, int64_t rows, int C, uint8_t *__restrict__ codes,
                float *__restrict__ scale) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = (int64_t(gridDim.x) * blockDim.x) >> 5;
    for (int64_t r = warp; r < rows; r += nwarps) {
        const float *f = in + r * C;
        float mx = 0.f;
        for (int c = lane; c < C; c += 32) mx = fmaxf(mx, fabsf(f[c]));
        for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        const float s = mx > 0.f ? __fdiv_rn(mx, 448.0f) : 1.0f;
        if (lane == 0) scale[r] = s;
        uint8_t *q = codes + r * C;
        for (int c = lane; c < C; c += 32)
            q[c] = uint8_t(__nv_cvt_float_to_fp8(__fdiv_rn(f[c], s), __NV_SATFINITE, __NV_E4M3));
    }
}

int grid_for(int64_t work, int threads) {
    int dev = 0, sms = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t want = (work + threads - 1) / threads;
    return int(want < 1 ? 1 : (want > int64_t(sms) * 8 ? int64_t(sms) * 8 : want));
}

}  // namespace
}  // namespace qr

using namespace qr;

extern "C" qr_status qr_quantize_bf16(const float *in, int64_t count, uint16_t *out,
                                      qr_stream stream) {
    if (count < 0 || (count > 0 && (!in || !out))) return QR_ERR_INVALID_ARG;
    if (count == 0) return QR_OK;
    bf16_kernel<<<grid_for(count, 256), 256, 0, reinterpret_cast<cudaStream_t>(stream)>>>(in, count, out);
    count_launch();
    return cudaGetLastError() == cudaSuccess ? QR_OK : QR_ERR_CUDA;
}

extern "C" qr_status qr_quantize_fp8(const float *in, int64_t rows, int32_t C, uint8_t *codes,
                                     float *scale, qr_stream stream) {
    if (rows < 0 || C < 1 || (rows > 0 && (!in || !codes || !scale))) return QR_ERR_INVALID_ARG;
    if (rows == 0) return QR_OK;
    fp8_rows_kernel<<<grid_for(rows * 32, 256), 256, 0, reinterpret_cast<cudaStream_t>(stream)>>>(
        in, rows, C, codes, scale);
    count_launch();
    return cudaGetLastError() == cudaSuccess ? QR_OK : QR_ERR_CUDA;
}
