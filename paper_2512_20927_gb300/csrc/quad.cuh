// Quads: the unit in which the blend kernels (blend.cu, batch.cu) read
// feature rows and write the map.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp8.h>

#include "qr_internal.cuh"

namespace qr {

// Four consecutive channels of a row ("a quad"): 16 bytes of F32, 8 of BF16,
// 4 of FP8.  Lane l of a warp owns quads l, l + 32, ... of a row, so every
// warp-wide row load reads 512, 256 or 128 contiguous bytes and every
// warp-wide store of the map writes 512 contiguous bytes, whatever the dtype.
template <int DT> struct Quad;
template <> struct Quad<QR_F32> { using T = uint4; static constexpr int B = 16; };
template <> struct Quad<QR_BF16> { using T = uint2; static constexpr int B = 8; };
template <> struct Quad<QR_FP8E4M3> { using T = uint32_t; static constexpr int B = 4; };

template <int DT>
__device__ __forceinline__ typename Quad<DT>::T ld_quad(const unsigned char *p) {
    if constexpr (DT == QR_F32) {
        uint4 r;
        asm volatile("ld.global.nc.v4.u32 {%0,%1,%2,%3}, [%4];"
                     : "=r"(r.x), "=r"(r.y), "=r"(r.z), "=r"(r.w) : "l"(p));
        return r;
    } else if constexpr (DT == QR_BF16) {
        uint2 r;
        asm volatile("ld.global.nc.v2.u32 {%0,%1}, [%2];" : "=r"(r.x), "=r"(r.y) : "l"(p));
        return r;
    } else {
        uint32_t r;
        asm volatile("ld.global.nc.u32 %0, [%1];" : "=r"(r) : "l"(p));
        return r;
    }
}
template <int DT>
__device__ __forceinline__ typename Quad<DT>::T zero_quad() {
    if constexpr (DT == QR_F32) return make_uint4(0, 0, 0, 0);
    else if constexpr (DT == QR_BF16) return make_uint2(0, 0);
    else return 0u;
}
// Exact widening to FP32 (BF16 by bit shifts, E4M3 by the conversion
// instructions; the per-Gaussian FP8 scale is applied to the weight).
template <int DT>
__device__ __forceinline__ void dec_quad(const typename Quad<DT>::T v, float *o) {
    if constexpr (DT == QR_F32) {
        o[0] = __uint_as_float(v.x); o[1] = __uint_as_float(v.y);
        o[2] = __uint_as_float(v.z); o[3] = __uint_as_float(v.w);
    } else if constexpr (DT == QR_BF16) {
        o[0] = __uint_as_float(v.x << 16); o[1] = __uint_as_float(v.x & 0xFFFF0000u);
        o[2] = __uint_as_float(v.y << 16); o[3] = __uint_as_float(v.y & 0xFFFF0000u);
    } else {
        const __half2_raw lo = __nv_cvt_fp8x2_to_halfraw2(__nv_fp8x2_storage_t(v & 0xFFFFu), __NV_E4M3);
        const __half2_raw hi = __nv_cvt_fp8x2_to_halfraw2(__nv_fp8x2_storage_t(v >> 16), __NV_E4M3);
        const float2 a = __half22float2(*reinterpret_cast<const __half2 *>(&lo));
        const float2 b = __half22float2(*reinterpret_cast<const __half2 *>(&hi));
        o[0] = a.x; o[1] = a.y; o[2] = b.x; o[3] = b.y;
    }
}

}  // namespace qr
