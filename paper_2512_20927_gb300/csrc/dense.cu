// K6: dense alpha compositing, Eq. 1 of the paper (V-Render, the plain method
// Q-Render is compared against):
//     out[p] = sum_i T_i alpha'_i f_i,   T_i = prod_{j<i} (1 - alpha'_j)
// over the pixel's whole depth-ordered list, with the same alpha' rules as the
// selection and a stop before the Gaussian whose test transmittance would
// fall below T_min.
//
// GB300 design: every pixel of a tile walks the same list, so the blend is a
// dense product W (pixels x batch) * F (batch x channels) per batch of 32
// list entries.  One CTA owns a screen tile and a 16/32/64-channel slice:
//   1. the batch's Gaussian records and feature-row slices are staged in
//      shared memory (coalesced 16-byte loads; BF16/FP8 widened here),
//   2. each thread walks its own pixel over the batch (scalar FP32, the exact
//      T recurrence) and writes the weights w = T alpha' to shared memory,
//   3. the accumulation runs as a register-tiled FP32 outer product (8 pixels
//      x 8 channels per thread for 64-channel slices), so every shared-memory
//      load feeds 8 FMAs.
// FP32 is kept on purpose: Eq. 1 is compared element by element with an FP64
// oracle, which a TF32/BF16 tensor-core product would not meet.
#include <cuda_bf16.h>
#include <cuda_fp8.h>

#include "qr_internal.cuh"

namespace qr {
namespace {

constexpr int kThreads = 256;
constexpr int kBatch = 32;

template <int DT>
__device__ __forceinline__ void widen16(const uint4 v, float scale, float *o);

template <>
__device__ __forceinline__ void widen16<QR_F32>(const uint4 v, float, float *o) {
    o[0] = __uint_as_float(v.x); o[1] = __uint_as_float(v.y);
    o[2] = __uint_as_float(v.z); o[3] = __uint_as_float(v.w);
}
template <>
__device__ __forceinline__ void widen16<QR_BF16>(const uint4 v, float, float *o) {
    const uint32_t u[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        o[2 * i] = __uint_as_float(u[i] << 16);
        o[2 * i + 1] = __uint_as_float(u[i] & 0xFFFF0000u);
    }
}
template <>
__device__ __forceinline__ void widen16<QR_FP8E4M3>(const uint4 v, float scale, float *o) {
    const uint32_t u[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const __half2_raw lo = __nv_cvt_fp8x2_to_halfraw2(__nv_fp8x2_storage_t(u[i] & 0xFFFFu), __NV_E4M3);
        const __half2_raw hi = __nv_cvt_fp8x2_to_halfraw2(__nv_fp8x2_storage_t(u[i] >> 16), __NV_E4M3);
        const float2 a = __half22float2(*reinterpret_cast<const __half2 *>(&lo));
        const float2 b = __half22float2(*reinterpret_cast<const __half2 *>(&hi));
        o[4 * i] = a.x * scale; o[4 * i + 1] = a.y * scale;
        o[4 * i + 2] = b.x * scale; o[4 * i + 3] = b.y * scale;
    }
}
template <int DT> struct Cpv;
template <> struct Cpv<QR_F32> { static constexpr int v = 4; };
template <> struct Cpv<QR_BF16> { static constexpr int v = 8; };
template <> struct Cpv<QR_FP8E4M3> { static constexpr int v = 16; };

// CC channels per CTA; thread tile PX x CH with (256/PX) * (CC/CH) == 256.
template <int DT, int CC, int PX, int CH>
__global__ void __launch_bounds__(kThreads)
dense_kernel(const float4 *__restrict__ rec_m, const float4 *__restrict__ rec_w,
              const float *__restrict__ rec_a, const float *__restrict__ rec_h,
             const uint32_t *__restrict__ isect_gid, const uint2 *__restrict__ ranges,
             const unsigned char *__restrict__ feat, const float *__restrict__ fscale, int C,
             int W, int H, int tile_w, int tiles_x, float alpha_min, float alpha_max,
             float T_min, float *__restrict__ out, float *__restrict__ T_final) {
    static_assert((kThreads / PX) * (CC / CH) == kThreads, "thread tile");
    constexpr int CPV = Cpv<DT>::v;
    constexpr int ESZ = DT == QR_F32 ? 4 : DT == QR_BF16 ? 2 : 1;
    __shared__ float4 s_m[kBatch];
    __shared__ float4 s_c[kBatch];
    __shared__ float s_a[kBatch];
    __shared__ float s_h[kBatch];
    __shared__ __align__(16) float s_F[kBatch][CC];
    __shared__ __align__(16) float s_W[kBatch][kThreads];

    const int tile = blockIdx.x;
    const int c0 = blockIdx.y * CC;
    const int tx = tile % tiles_x, ty = tile / tiles_x;
    const int tile_h = kThreads / tile_w;
    const int lx = threadIdx.x % tile_w, ly = threadIdx.x / tile_w;
    const int px = tx * tile_w + lx, py = ty * tile_h + ly;
    const bool inside = px < W && py < H;
    const float ux = float(px) + 0.5f, uy = float(py) + 0.5f;
    const uint2 range = ranges[tile];

    // GEMM roles
    constexpr int PG = kThreads / PX;  // pixel groups
    const int pg = threadIdx.x % PG, cg = threadIdx.x / PG;
    float acc[PX][CH];
#pragma unroll
    for (int i = 0; i < PX; ++i)
#pragma unroll
        for (int j = 0; j < CH; ++j) acc[i][j] = 0.f;

    float T = 1.0f;
    bool done = !inside;
    const size_t row_bytes = size_t(C) * ESZ;

    for (uint32_t b = range.x; b < range.y; b += kBatch) {
        if (__syncthreads_count(done) == kThreads) break;
        const int nb = int(min(uint32_t(kBatch), range.y - b));
        // stage records and feature slices
        if (threadIdx.x < nb) {
            const uint32_t g = isect_gid[b + threadIdx.x];
            s_m[threadIdx.x] = rec_m[g];
            s_c[threadIdx.x] = rec_w[g];
            s_a[threadIdx.x] = rec_a[g];
            s_h[threadIdx.x] = rec_h[g];
        }
        constexpr int VPR = CC / CPV;  // 16-byte vectors per row slice
        for (int i = threadIdx.x; i < kBatch * VPR; i += kThreads) {
            const int r = i / VPR, v = i % VPR;
            float tmp[CPV];
            if (r < nb) {
                const uint32_t g = isect_gid[b + r];
                const uint4 x = *reinterpret_cast<const uint4 *>(feat + size_t(g) * row_bytes +
                                                                 size_t(c0 + v * CPV) * ESZ);
                widen16<DT>(x, DT == QR_FP8E4M3 ? fscale[g] : 1.f, tmp);
            } else {
#pragma unroll
                for (int q = 0; q < CPV; ++q) tmp[q] = 0.f;
            }
#pragma unroll
            for (int q = 0; q < CPV; ++q) s_F[r][v * CPV + q] = tmp[q];
        }
        __syncthreads();
        // weights: thread = pixel, exact T recurrence
        for (int j = 0; j < kBatch; ++j) {
            float w = 0.f;
            if (!done && j < nb) {
                const float4 mm = s_m[j];
                const float4 cc = s_c[j];
                const PixelTerm pt = eval_half_q(ux, uy, mm, cc);
                const float a = pt.half_q > s_h[j] ? 0.f : eval_alpha(s_a[j], pt.half_q, alpha_max);
                if (a >= alpha_min) {
                    const float Tt = T * (1.0f - a);
                    if (T_min > 0.f && Tt < T_min) {
                        done = true;
                    } else {
                        w = T * a;
                        T = Tt;
                    }
                }
            }
            s_W[j][threadIdx.x] = w;
        }
        __syncthreads();
        // accumulate: acc[px][ch] += W[j][px] * F[j][ch]
        for (int j = 0; j < nb; ++j) {
            float wv[PX], fv[CH];
            if constexpr (PX % 4 == 0) {
#pragma unroll
                for (int i = 0; i < PX; i += 4) {
                    const float4 t = *reinterpret_cast<const float4 *>(&s_W[j][pg * PX + i]);
                    wv[i] = t.x; wv[i + 1] = t.y; wv[i + 2] = t.z; wv[i + 3] = t.w;
                }
            } else {
#pragma unroll
                for (int i = 0; i < PX; ++i) wv[i] = s_W[j][pg * PX + i];
            }
#pragma unroll
            for (int i = 0; i < CH; i += 4) {
                const float4 t = *reinterpret_cast<const float4 *>(&s_F[j][cg * CH + i]);
                fv[i] = t.x; fv[i + 1] = t.y; fv[i + 2] = t.z; fv[i + 3] = t.w;
            }
#pragma unroll
            for (int a = 0; a < PX; ++a)
#pragma unroll
                for (int c = 0; c < CH; ++c) acc[a][c] = fmaf(wv[a], fv[c], acc[a][c]);
        }
    }
    // write the slice
#pragma unroll
    for (int a = 0; a < PX; ++a) {
        const int t = pg * PX + a;
        const int qx = tx * tile_w + t % tile_w, qy = ty * tile_h + t / tile_w;
        if (qx < W && qy < H) {
            float *o = out + (int64_t(qy) * W + qx) * C + c0 + cg * CH;
#pragma unroll
            for (int c = 0; c < CH; c += 4)
                *reinterpret_cast<float4 *>(o + c) =
                    make_float4(acc[a][c], acc[a][c + 1], acc[a][c + 2], acc[a][c + 3]);
        }
    }
    if (T_final && blockIdx.y == 0 && inside) T_final[int64_t(py) * W + px] = T;
}

template <int DT, int CC, int PX, int CH>
cudaError_t run(const qr_frame &f, const void *feat, const float *scale, int C, float *out,
                float *T_final, cudaStream_t s) {
    dim3 grid(unsigned(num_tiles(f)), unsigned(C / CC));
    dense_kernel<DT, CC, PX, CH><<<grid, kThreads, 0, s>>>(
        slot<float4>(f, S_REC_M), slot<float4>(f, S_REC_C), slot<float>(f, S_REC_A), slot<float>(f, S_REC_H),
        slot<uint32_t>(f, S_IGID),
        slot<uint2>(f, S_RANGES), static_cast<const unsigned char *>(feat), scale, C, f.camera.width,
        f.camera.height, f.params.tile_w, f.tiles_x, f.params.alpha_min, f.params.alpha_max,
        f.params.T_min, out, T_final);
    count_launch();
    return cudaGetLastError();
}

template <int DT>
cudaError_t dispatch(const qr_frame &f, const void *feat, const float *scale, int C, float *out,
                     float *T_final, cudaStream_t s) {
    constexpr int cpv = Cpv<DT>::v;
    if (C % 64 == 0) return run<DT, 64, 8, 8>(f, feat, scale, C, out, T_final, s);
    if (C % 32 == 0) return run<DT, 32, 8, 4>(f, feat, scale, C, out, T_final, s);
    if (C % 16 == 0) return run<DT, 16, 4, 4>(f, feat, scale, C, out, T_final, s);
    if constexpr (cpv <= 8)
        if (C % 8 == 0) return run<DT, 8, 2, 4>(f, feat, scale, C, out, T_final, s);
    if constexpr (cpv <= 4)
        if (C % 4 == 0) return run<DT, 4, 1, 4>(f, feat, scale, C, out, T_final, s);
    return cudaErrorInvalidValue;
}

}  // namespace

bool dense_supported(qr_dtype dt, int C) {
    const int cpv = dt == QR_F32 ? 4 : dt == QR_BF16 ? 8 : 16;
    return C > 0 && C % cpv == 0;
}

cudaError_t launch_dense(const qr_frame &f, const void *feat, const float *scale, qr_dtype dt,
                         int C, float *out, float *T_final, cudaStream_t s) {
    if (num_tiles(f) == 0) return cudaSuccess;
    switch (dt) {
        case QR_F32: return dispatch<QR_F32>(f, feat, scale, C, out, T_final, s);
        case QR_BF16: return dispatch<QR_BF16>(f, feat, scale, C, out, T_final, s);
        case QR_FP8E4M3: return dispatch<QR_FP8E4M3>(f, feat, scale, C, out, T_final, s);
    }
    return cudaErrorInvalidValue;
}

}  // namespace qr
