// K5b: the blend half of Algorithm 1 (Sec. 4.2, "alpha-blending on quantile
// Gaussians" and "normalizing feature vector"):
//     out[p] = sum_{j < cnt[p]} w[p][j] * f[ids[p][j]]
// with the 1/(1 - T^Q) normalisation already folded into w by the selection.
//
// GB300 design: this is the bandwidth-bound stage (about zero flops per byte),
// so the kernel is built around 16-byte vector traffic:
//   - one warp per pixel (for rows of 512 B or more; narrower rows pack
//     several pixels into a warp), each lane owning a fixed set of 16-byte
//     column vectors of the row, so every warp-wide load or store moves 512
//     contiguous bytes;
//   - the pixel's ids and weights are read at one address by all of its
//     lanes (a single L1 broadcast per entry);
//   - all row loads of a pixel are issued before the FMAs (unrolled by 4
//     rows) to keep enough bytes in flight per SM;
//   - BF16 rows are widened with bit shifts, FP8 E4M3 rows with the hardware
//     conversion instructions; FP8 rows fold their per-Gaussian scale into
//     the weight;
//   - the map is written with streaming (evict-first) 16-byte stores so it
//     does not displace the feature rows that neighbouring pixels share in L2;
//   - one CTA renders one 16x16 screen tile, its warps interleaved over the
//     tile's pixels, so rows shared by a tile's pixels are re-read from the
//     SM's L1 instead of L2.
#include <cuda_bf16.h>
#include <cuda_fp8.h>

#include "qr_internal.cuh"
#include "quad.cuh"

namespace qr {
namespace {

constexpr int kThreads = 256;

// Channels carried by one 16-byte vector of a row.
template <int DT> struct Vec;
template <> struct Vec<QR_F32> { static constexpr int C = 4; };
template <> struct Vec<QR_BF16> { static constexpr int C = 8; };
template <> struct Vec<QR_FP8E4M3> { static constexpr int C = 16; };

// acc[0..1] += w * (x0, x1) with one packed FP32x2 FMA (each lane of the pair
// rounds exactly like a scalar fmaf).
__device__ __forceinline__ void fma2(float *acc, float w, float x0, float x1) {
    asm("{\n .reg .b64 a, ww, xx;\n mov.b64 a, {%0, %1};\n mov.b64 ww, {%2, %2};\n"
        " mov.b64 xx, {%3, %4};\n fma.rn.f32x2 a, ww, xx, a;\n mov.b64 {%0, %1}, a;\n}\n"
        : "+f"(acc[0]), "+f"(acc[1]) : "f"(w), "f"(x0), "f"(x1));
}

template <int DT>
__device__ __forceinline__ void decode_fma(const uint4 v, float w, float *acc);

template <>
__device__ __forceinline__ void decode_fma<QR_F32>(const uint4 v, float w, float *acc) {
    fma2(acc + 0, w, __uint_as_float(v.x), __uint_as_float(v.y));
    fma2(acc + 2, w, __uint_as_float(v.z), __uint_as_float(v.w));
}

__device__ __forceinline__ void bf16x2_fma(uint32_t u, float w, float *acc) {
    fma2(acc, w, __uint_as_float(u << 16), __uint_as_float(u & 0xFFFF0000u));
}

template <>
__device__ __forceinline__ void decode_fma<QR_BF16>(const uint4 v, float w, float *acc) {
    bf16x2_fma(v.x, w, acc + 0);
    bf16x2_fma(v.y, w, acc + 2);
    bf16x2_fma(v.z, w, acc + 4);
    bf16x2_fma(v.w, w, acc + 6);
}

__device__ __forceinline__ void fp8x4_fma(uint32_t u, float w, float *acc) {
    const __half2_raw lo = __nv_cvt_fp8x2_to_halfraw2(__nv_fp8x2_storage_t(u & 0xFFFFu), __NV_E4M3);
    const __half2_raw hi = __nv_cvt_fp8x2_to_halfraw2(__nv_fp8x2_storage_t(u >> 16), __NV_E4M3);
    const float2 a = __half22float2(*reinterpret_cast<const __half2 *>(&lo));
    const float2 b = __half22float2(*reinterpret_cast<const __half2 *>(&hi));
    fma2(acc + 0, w, a.x, a.y);
    fma2(acc + 2, w, b.x, b.y);
}

template <>
__device__ __forceinline__ void decode_fma<QR_FP8E4M3>(const uint4 v, float w, float *acc) {
    fp8x4_fma(v.x, w, acc + 0);
    fp8x4_fma(v.y, w, acc + 4);
    fp8x4_fma(v.z, w, acc + 8);
    fp8x4_fma(v.w, w, acc + 12);
}

// A 16-byte vector widened to FP32 once (exact for BF16 and E4M3), so that a
// row shared by several pixels is decoded once and FMA'd into each of them.
template <int DT>
__device__ __forceinline__ void decode_vec(const uint4 v, float *o) {
    if constexpr (DT == QR_F32) {
        o[0] = __uint_as_float(v.x); o[1] = __uint_as_float(v.y);
        o[2] = __uint_as_float(v.z); o[3] = __uint_as_float(v.w);
    } else if constexpr (DT == QR_BF16) {
        const uint32_t u[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            o[2 * i] = __uint_as_float(u[i] << 16);
            o[2 * i + 1] = __uint_as_float(u[i] & 0xFFFF0000u);
        }
    } else {
        const uint32_t u[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const __half2_raw lo = __nv_cvt_fp8x2_to_halfraw2(__nv_fp8x2_storage_t(u[i] & 0xFFFFu), __NV_E4M3);
            const __half2_raw hi = __nv_cvt_fp8x2_to_halfraw2(__nv_fp8x2_storage_t(u[i] >> 16), __NV_E4M3);
            const float2 a = __half22float2(*reinterpret_cast<const __half2 *>(&lo));
            const float2 b = __half22float2(*reinterpret_cast<const __half2 *>(&hi));
            o[4 * i] = a.x; o[4 * i + 1] = a.y; o[4 * i + 2] = b.x; o[4 * i + 3] = b.y;
        }
    }
}

// acc[0..N) += w * f[0..N) in packed pairs (each half rounds like fmaf)
template <int N>
__device__ __forceinline__ void fma_vec(const float *f, float w, float *acc) {
#pragma unroll
    for (int i = 0; i < N; i += 2) fma2(acc + i, w, f[i], f[i + 1]);
}

__device__ __forceinline__ uint4 ld_row(const uint4 *p) {
    uint4 r;
    asm volatile("ld.global.nc.v4.u32 {%0,%1,%2,%3}, [%4];"
                 : "=r"(r.x), "=r"(r.y), "=r"(r.z), "=r"(r.w) : "l"(p));
    return r;
}

__device__ __forceinline__ void st_stream(float4 *p, float4 v) {
    asm volatile("st.global.cs.v4.f32 [%0], {%1,%2,%3,%4};"
                 :: "l"(p), "f"(v.x), "f"(v.y), "f"(v.z), "f"(v.w) : "memory");
}

// Pixel visited by work item `item` in screen-tile order (16x16 tiles).
__device__ __forceinline__ int64_t tile_order_pixel(int64_t item, int W, int H) {
    if (W <= 0) return item;
    const int tiles_x = (W + 15) >> 4;
    const int64_t t = item >> 8;
    const int r = int(item & 255);
    const int tx = int(t % tiles_x), ty = int(t / tiles_x);
    const int x = tx * 16 + (r & 15), y = ty * 16 + (r >> 4);
    if (x >= W || y >= H) return -1;
    return int64_t(y) * W + x;
}

// LPP lanes per pixel, VPL 16-byte vectors per lane; row = LPP*VPL vectors.
template <int DT, int LPP, int VPL>
__global__ void __launch_bounds__(kThreads)
blend_kernel(const uint4 *__restrict__ feat, const float *__restrict__ scale, int64_t n_gauss,
             const int32_t *__restrict__ ids, const float *__restrict__ wts,
             const uint8_t *__restrict__ cnt, int64_t P, int K, int W, int H,
             float4 *__restrict__ out) {
    pdl_wait();   // the predecessor's outputs are complete and visible
    constexpr int CPV = Vec<DT>::C;          // channels per vector
    constexpr int PPW = 32 / LPP;            // pixels per warp
    constexpr int ROWV = LPP * VPL;          // vectors per row
    const int lane = threadIdx.x & 31;
    const int sub = lane / LPP, sl = lane % LPP;
    const int64_t items = (W > 0) ? int64_t((W + 15) >> 4) * ((H + 15) >> 4) * 256 : P;
    const int warp = threadIdx.x >> 5;
    const int64_t chunk0 = int64_t(blockIdx.x) * 256;   // one 16x16 screen tile per CTA
    for (int it = warp * PPW + sub; it < 256; it += (kThreads / 32) * PPW) {
        const int64_t item = chunk0 + it;
        const int64_t p = (item < items) ? tile_order_pixel(item, W, H) : -1;
        const int c = (p >= 0) ? int(cnt[p]) : 0;
        const int32_t *pid = ids + p * K;
        const float *pw = wts + p * K;
        float acc[VPL][CPV];
#pragma unroll
        for (int v = 0; v < VPL; ++v)
#pragma unroll
            for (int q = 0; q < CPV; ++q) acc[v][q] = 0.f;
        for (int j0 = 0; j0 < c; j0 += 4) {
            uint4 r[4][VPL];
            float wj[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int j = j0 + u;
                const bool ok = j < c;
                int id = ok ? pid[j] : 0;     // same address across the pixel's lanes: one L1 broadcast
                float w = ok ? pw[j] : 0.f;
                if (uint64_t(int64_t(id)) >= uint64_t(n_gauss)) { id = 0; w = 0.f; }
                if (DT == QR_FP8E4M3 && ok) w *= scale[id];
                wj[u] = w;
                const uint4 *row = feat + int64_t(id) * ROWV + sl;
#pragma unroll
                for (int v = 0; v < VPL; ++v)
                    r[u][v] = ok ? ld_row(row + v * LPP) : make_uint4(0, 0, 0, 0);
            }
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int v = 0; v < VPL; ++v) decode_fma<DT>(r[u][v], wj[u], acc[v]);
        }
        if (p >= 0) {
            float4 *o = out + p * (int64_t(ROWV) * CPV / 4);
#pragma unroll
            for (int v = 0; v < VPL; ++v)
#pragma unroll
                for (int q = 0; q < CPV / 4; ++q)
                    st_stream(o + int64_t(sl + v * LPP) * (CPV / 4) + q,
                              make_float4(acc[v][4 * q], acc[v][4 * q + 1], acc[v][4 * q + 2],
                                          acc[v][4 * q + 3]));
        }
    }
}

// Wide rows (one warp per row): a warp owns a group of G neighbouring pixels
// (2x2 for G = 4, 2x1 for G = 2) whose selections are subsequences of the same
// tile list and mostly share rows.  Lane g*K + j holds entry j of pixel g;
// __match_any_sync groups equal ids and each distinct row is loaded once and
// accumulated into every pixel of the group with that pixel's weight (zero
// weights are skipped).  L1 row traffic drops from sum(counts) to the number
// of distinct rows of the group.
template <int G>
__device__ __forceinline__ int64_t group_pixel(int64_t chunk0, int gi, int m, int W, int H,
                                               int64_t items) {
    int r;
    if (G == 4) {
        const int qx = gi & 7, qy = gi >> 3;
        r = (2 * qy + (m >> 1)) * 16 + 2 * qx + (m & 1);
    } else if (G == 2) {
        r = (gi >> 3) * 16 + 2 * (gi & 7) + m;
    } else {
        r = gi;
    }
    const int64_t item = chunk0 + r;
    if (item >= items) return -1;
    return tile_order_pixel(item, W, H);
}

// The G weights of each distinct row are gathered once into a shared-memory
// table (slot = rank of the row's leader lane, one float per pixel; a pixel
// that lists an id twice gets the sum), so the row loop reads them with one
// broadcast load instead of a chain of shuffles.
//
// Rows are handled in quads (above): QPL quads per lane per channel chunk, NCH
// chunks per row (a work item is a (pixel group, chunk) pair; NCH > 1 means
// fewer accumulators per thread and more warps per item).  The next item's
// counts, ids and weights are loaded (three independent loads) before the
// current item's rows, U rows are in flight per step (64-128 bytes per lane),
// and FP8 rows load their per-Gaussian scale beside the row and apply it to
// the row's weights, so no load waits on another's result.  An FP8 row's
// weight for a pixel is (the pixel's weight for it) * scale, rounded once: a
// selection lists a Gaussian at most once per pixel.
template <int DT, int QPL, int G, int NCH>
__global__ void __launch_bounds__(kThreads)
blend_group_kernel(const unsigned char *__restrict__ feat, const float *__restrict__ scale,
                   int64_t n_gauss, const int32_t *__restrict__ ids,
                   const float *__restrict__ wts, const uint8_t *__restrict__ cnt, int64_t P,
                   int K, int W, int H, float4 *__restrict__ out) {
    pdl_wait();   // the predecessor's outputs are complete and visible
    constexpr int QB = Quad<DT>::B;
    constexpr int CQ = 32 * QPL;             // quads of a chunk
    constexpr int ROWQ = CQ * NCH;           // quads of a row (C / 4)
    constexpr int U = (QPL * QB >= 64) ? 2 : (QPL * QB >= 32 ? 128 / (QPL * QB) : 4);
    constexpr unsigned FULL = 0xffffffffu;
    constexpr int NW = kThreads / 32;
    constexpr int NITEMS = (256 / G) * NCH;
    __shared__ __align__(16) float s_w[NW][32][G];
    __shared__ int s_id[NW][32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t items = (W > 0) ? int64_t((W + 15) >> 4) * ((H + 15) >> 4) * 256 : P;
    const int64_t chunk0 = int64_t(blockIdx.x) * 256;
    const int m = lane / K, j = lane - m * K;
    auto fetch = [&](int gi, int64_t &p, int &idr, float &wr, int &c) {
        p = -1;
        if (m < G) p = (W > 0) ? group_pixel<G>(chunk0, gi, m, W, H, items)
                               : (chunk0 + gi * G + m < items ? chunk0 + gi * G + m : -1);
        idr = -1;
        wr = 0.f;
        c = 0;
        if (p >= 0) {
            c = int(cnt[p]);
            idr = ids[p * K + j];
            wr = wts[p * K + j];
        }
    };
    int64_t p;
    int idr, c;
    float wr;
    fetch(warp / NCH, p, idr, wr, c);
    for (int it = warp; it < NITEMS; it += NW) {
        const int ch = it % NCH;
        const bool ok = p >= 0 && j < c && uint64_t(int64_t(idr)) < uint64_t(n_gauss);
        const int id = ok ? idr : -1;
        const float w = ok ? wr : 0.f;
        const int64_t pc = p;
        if (it + NW < NITEMS) fetch((it + NW) / NCH, p, idr, wr, c);
        const unsigned peers = __match_any_sync(FULL, id);
        const int leader = __ffs(peers) - 1;
        const unsigned leaders = __ballot_sync(FULL, id >= 0 && lane == leader);
        const int nrows = __popc(leaders);
#pragma unroll
        for (int g = 0; g < G; ++g) s_w[warp][lane][g] = 0.f;
        __syncwarp();
        if (id >= 0) {
            const int slot = __popc(leaders & ((1u << leader) - 1u));
            atomicAdd(&s_w[warp][slot][m], w);   // m < G for every listed entry
            if (lane == leader) s_id[warp][slot] = id;
        }
        __syncwarp();
        float acc[G][QPL][4];
#pragma unroll
        for (int g = 0; g < G; ++g)
#pragma unroll
            for (int v = 0; v < QPL; ++v)
#pragma unroll
                for (int q = 0; q < 4; ++q) acc[g][v][q] = 0.f;
        const unsigned char *fch = feat + size_t(ch * CQ + lane) * QB;
        for (int r0 = 0; r0 < nrows; r0 += U) {
            typename Quad<DT>::T r[U][QPL];
            float sc[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const bool ok = r0 + u < nrows;
                const int rid = ok ? s_id[warp][r0 + u] : 0;
                const unsigned char *row = fch + size_t(rid) * (size_t(ROWQ) * QB);
#pragma unroll
                for (int v = 0; v < QPL; ++v)
                    r[u][v] = ok ? ld_quad<DT>(row + size_t(32 * v) * QB) : zero_quad<DT>();
                if (DT == QR_FP8E4M3) sc[u] = ok ? scale[rid] : 0.f;
            }
#pragma unroll
            for (int u = 0; u < U; ++u) {
                if (r0 + u >= nrows) break;
                float wg[G];
#pragma unroll
                for (int g = 0; g < G; ++g)
                    wg[g] = DT == QR_FP8E4M3 ? s_w[warp][r0 + u][g] * sc[u] : s_w[warp][r0 + u][g];
                float fv[QPL][4];
#pragma unroll
                for (int v = 0; v < QPL; ++v) dec_quad<DT>(r[u][v], fv[v]);
#pragma unroll
                for (int g = 0; g < G; ++g)
                    if (wg[g] != 0.f) {
#pragma unroll
                        for (int v = 0; v < QPL; ++v) fma_vec<4>(fv[v], wg[g], acc[g][v]);
                    }
            }
        }
#pragma unroll
        for (int g = 0; g < G; ++g) {
            const int64_t pg = __shfl_sync(FULL, pc, g * K < 32 ? g * K : 0);
            if (pg >= 0) {
                float4 *o = out + pg * int64_t(ROWQ) + ch * CQ + lane;
#pragma unroll
                for (int v = 0; v < QPL; ++v)
                    st_stream(o + 32 * v, make_float4(acc[g][v][0], acc[g][v][1], acc[g][v][2],
                                                      acc[g][v][3]));
            }
        }
        __syncwarp();   // the table is rewritten by the next item
    }
}

// Channel chunks a row of QT quads per lane is split into by default: the
// fewest that keep at most 4 quads (16 accumulators per pixel) per lane.
template <int QT>
constexpr int default_chunks() {
    return QT <= 4 ? 1 : QT % 4 == 0 ? QT / 4 : QT % 3 == 0 ? QT / 3 : QT / 2;
}

int g_blend_chunks = 0;   // qr_set_blend_chunks: 0 = default_chunks

template <int DT, int QT, int G, int NCH>
cudaError_t go_group(const void *feat, const float *scale, int64_t n_gauss, const int32_t *ids,
                     const float *w, const uint8_t *cnt, int64_t P, int K, int W, int H,
                     float *out, cudaStream_t s) {
    const int64_t items = (W > 0) ? int64_t((W + 15) >> 4) * ((H + 15) >> 4) * 256 : P;
    const unsigned blocks = unsigned((items + 255) / 256);
    return pdl_launch(blend_group_kernel<DT, QT / NCH, G, NCH>, dim3(blocks), dim3(kThreads), 0, s,
                      static_cast<const unsigned char *>(feat), scale, n_gauss, ids, w, cnt, P, K,
                      W, H, reinterpret_cast<float4 *>(out));
}

// QT = C / 128 quads per lane over the whole row (e.g. 4 for 512-D rows of
// any dtype).  With K <= 8 (pixel groups of 4) and QT = 4 the chunk count can
// be chosen (qr_set_blend_chunks: 1, 2 or 4); the results are the same for
// every choice.
template <int DT, int QT>
cudaError_t run_group(const void *feat, const float *scale, int64_t n_gauss, const int32_t *ids,
                      const float *w, const uint8_t *cnt, int64_t P, int K, int W, int H,
                      float *out, cudaStream_t s) {
    constexpr int DEF = default_chunks<QT>();
    cudaError_t e;
    if (K <= 8) {
        const int want = g_blend_chunks > 0 ? g_blend_chunks : DEF;
        if constexpr (QT == 4) {
            if (want == 2)
                e = go_group<DT, QT, 4, 2>(feat, scale, n_gauss, ids, w, cnt, P, K, W, H, out, s);
            else if (want == 4)
                e = go_group<DT, QT, 4, 4>(feat, scale, n_gauss, ids, w, cnt, P, K, W, H, out, s);
            else
                e = go_group<DT, QT, 4, 1>(feat, scale, n_gauss, ids, w, cnt, P, K, W, H, out, s);
        } else {
            e = go_group<DT, QT, 4, DEF>(feat, scale, n_gauss, ids, w, cnt, P, K, W, H, out, s);
        }
    } else if (K <= 16) {
        e = go_group<DT, QT, 2, DEF>(feat, scale, n_gauss, ids, w, cnt, P, K, W, H, out, s);
    } else {
        e = go_group<DT, QT, 1, DEF>(feat, scale, n_gauss, ids, w, cnt, P, K, W, H, out, s);
    }
    count_launch();
    return e != cudaSuccess ? e : cudaGetLastError();
}

template <int DT, int LPP, int VPL>
cudaError_t run(const void *feat, const float *scale, int64_t n_gauss, const int32_t *ids,
                const float *w, const uint8_t *cnt, int64_t P, int K, int W, int H, float *out,
                cudaStream_t s) {
    const int64_t items = (W > 0) ? int64_t((W + 15) >> 4) * ((H + 15) >> 4) * 256 : P;
    const int64_t blocks = (items + 255) / 256;
    const cudaError_t e = pdl_launch(blend_kernel<DT, LPP, VPL>, dim3(unsigned(blocks)), dim3(kThreads),
                                     0, s, static_cast<const uint4 *>(feat), scale, n_gauss, ids, w,
                                     cnt, P, K, W, H, reinterpret_cast<float4 *>(out));
    count_launch();
    return e != cudaSuccess ? e : cudaGetLastError();
}

template <int DT>
cudaError_t dispatch(const void *feat, const float *scale, int64_t n_gauss, int C,
                     const int32_t *ids, const float *w, const uint8_t *cnt, int64_t P, int K,
                     int W, int H, float *out, cudaStream_t s) {
    const int rowv = C / Vec<DT>::C;  // 16-byte vectors per row
    constexpr int CPV4 = Vec<DT>::C / 4;  // quads per 16-byte vector
    switch (rowv) {
        case 1: return run<DT, 1, 1>(feat, scale, n_gauss, ids, w, cnt, P, K, W, H, out, s);
        case 2: return run<DT, 2, 1>(feat, scale, n_gauss, ids, w, cnt, P, K, W, H, out, s);
        case 4: return run<DT, 4, 1>(feat, scale, n_gauss, ids, w, cnt, P, K, W, H, out, s);
        case 8: return run<DT, 8, 1>(feat, scale, n_gauss, ids, w, cnt, P, K, W, H, out, s);
        case 16: return run<DT, 16, 1>(feat, scale, n_gauss, ids, w, cnt, P, K, W, H, out, s);
        // wide rows: QT = C / 128 quads per lane
        case 32: return run_group<DT, CPV4 * 1>(feat, scale, n_gauss, ids, w, cnt, P, K, W, H, out, s);
        case 64: return run_group<DT, CPV4 * 2>(feat, scale, n_gauss, ids, w, cnt, P, K, W, H, out, s);
        case 96: return run_group<DT, CPV4 * 3>(feat, scale, n_gauss, ids, w, cnt, P, K, W, H, out, s);
        case 128: return run_group<DT, CPV4 * 4>(feat, scale, n_gauss, ids, w, cnt, P, K, W, H, out, s);
        case 256: return run<DT, 32, 8>(feat, scale, n_gauss, ids, w, cnt, P, K, W, H, out, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace

bool set_blend_chunks(int chunks) {
    if (chunks != 0 && chunks != 1 && chunks != 2 && chunks != 4) return false;
    g_blend_chunks = chunks;
    return true;
}

// Row widths the blend kernel is built for (16-byte vectors per row).
bool blend_supported(qr_dtype dt, int C) {
    const int cpv = dt == QR_F32 ? 4 : dt == QR_BF16 ? 8 : 16;
    if (C <= 0 || C % cpv) return false;
    const int rowv = C / cpv;
    return rowv == 1 || rowv == 2 || rowv == 4 || rowv == 8 || rowv == 16 || rowv == 32 ||
           rowv == 64 || rowv == 96 || rowv == 128 || rowv == 256;
}

cudaError_t launch_blend_tiled(const void *feat, const float *scale, qr_dtype dt, int C,
                               int64_t n_gauss, const int32_t *ids, const float *w,
                               const uint8_t *cnt, int64_t P, int K, int W, int H, float *out,
                               cudaStream_t s) {
    switch (dt) {
        case QR_F32: return dispatch<QR_F32>(feat, scale, n_gauss, C, ids, w, cnt, P, K, W, H, out, s);
        case QR_BF16: return dispatch<QR_BF16>(feat, scale, n_gauss, C, ids, w, cnt, P, K, W, H, out, s);
        case QR_FP8E4M3: return dispatch<QR_FP8E4M3>(feat, scale, n_gauss, C, ids, w, cnt, P, K, W, H, out, s);
    }
    return cudaErrorInvalidValue;
}

}  // namespace qr
