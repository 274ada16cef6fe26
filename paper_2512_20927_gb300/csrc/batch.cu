// Many views in one persistent launch: Algorithm 1's selection and blend fused
// per screen tile, over the tiles of every view of a batch (the paper renders
// 4 random training views per scene per step, Appendix D; inference renders
// many views of several scenes).
//
// GB300 design: a grid of (SMs x resident CTAs) persistent CTAs pulls
// (view, tile) work items from one atomic counter, so views of very different
// sizes balance without a host round trip.  For each tile:
//   1. selection (thread per pixel): the tile's depth-ordered list is staged
//      through shared memory 256 entries at a time; each warp culls the
//      staged entries against its box of pixel centres and walks only the
//      survivors, four per step, with the same alpha' evaluation and the same
//      Algorithm 1 rule as qr_select; the kept ids and normalised weights
//      stay in shared memory and are also written out (coalesced tile-row
//      runs) for a backward pass;
//   2. blend (warp per 2x2 / 2x1 pixel group, like qr_blend): equal ids of the
//      group are merged with __match_any_sync, the group's weights of each
//      distinct row are gathered into a per-warp shared-memory table, each
//      distinct feature row is read once with 16-byte loads and accumulated
//      into every pixel of the group, and the rows of the map are written
//      with streaming stores.
// Per-view descriptors live in device memory (qr_batch_prepare), the counter
// is cleared by a memset on the stream, so the launch can sit in a CUDA graph.
#include <cuda_bf16.h>
#include <cuda_fp8.h>

#include "qr_internal.cuh"

namespace qr {

struct BatchView {
    const float4 *rec_m;
    const float4 *rec_w;
    const float *rec_a;
    const float *rec_h;
    const uint32_t *igid;
    const uint2 *ranges;
    const unsigned char *feat;
    const float *fscale;
    int32_t *ids;
    float *w;
    uint8_t *cnt;
    float *out;
    int64_t n_gauss;
    int W, H, tile_w, tiles_x, tiles_y, K;
    float alpha_min, alpha_max;
    uint32_t tile_base;     // first work item of this view
    uint32_t pad;
};

namespace {

constexpr int T = 256;

template <int DT> struct VecT;
template <> struct VecT<QR_F32> { static constexpr int C = 4; };
template <> struct VecT<QR_BF16> { static constexpr int C = 8; };
template <> struct VecT<QR_FP8E4M3> { static constexpr int C = 16; };

__device__ __forceinline__ void fma2b(float *acc, float w, float x0, float x1) {
    asm("{\n .reg .b64 a, ww, xx;\n mov.b64 a, {%0, %1};\n mov.b64 ww, {%2, %2};\n"
        " mov.b64 xx, {%3, %4};\n fma.rn.f32x2 a, ww, xx, a;\n mov.b64 {%0, %1}, a;\n}\n"
        : "+f"(acc[0]), "+f"(acc[1]) : "f"(w), "f"(x0), "f"(x1));
}

template <int DT>
__device__ __forceinline__ void dec_fma(const uint4 v, float w, float *acc) {
    if constexpr (DT == QR_F32) {
        fma2b(acc + 0, w, __uint_as_float(v.x), __uint_as_float(v.y));
        fma2b(acc + 2, w, __uint_as_float(v.z), __uint_as_float(v.w));
    } else if constexpr (DT == QR_BF16) {
        const uint32_t u[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
        for (int i = 0; i < 4; ++i)
            fma2b(acc + 2 * i, w, __uint_as_float(u[i] << 16), __uint_as_float(u[i] & 0xFFFF0000u));
    } else {
        const uint32_t u[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const __half2_raw lo = __nv_cvt_fp8x2_to_halfraw2(__nv_fp8x2_storage_t(u[i] & 0xFFFFu), __NV_E4M3);
            const __half2_raw hi = __nv_cvt_fp8x2_to_halfraw2(__nv_fp8x2_storage_t(u[i] >> 16), __NV_E4M3);
            const float2 a = __half22float2(*reinterpret_cast<const __half2 *>(&lo));
            const float2 b = __half22float2(*reinterpret_cast<const __half2 *>(&hi));
            fma2b(acc + 4 * i, w, a.x, a.y);
            fma2b(acc + 4 * i + 2, w, b.x, b.y);
        }
    }
}

// A 16-byte vector widened to FP32 once (exact for BF16 and E4M3); the group
// loop then FMAs it into each pixel that lists the row.
template <int DT>
__device__ __forceinline__ void dec_vec(const uint4 v, float *o) {
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

__device__ __forceinline__ uint4 ldg_nc(const uint4 *p) {
    uint4 r;
    asm volatile("ld.global.nc.v4.u32 {%0,%1,%2,%3}, [%4];"
                 : "=r"(r.x), "=r"(r.y), "=r"(r.z), "=r"(r.w) : "l"(p));
    return r;
}

__device__ __forceinline__ void st_cs(float4 *p, float4 v) {
    asm volatile("st.global.cs.v4.f32 [%0], {%1,%2,%3,%4};"
                 :: "l"(p), "f"(v.x), "f"(v.y), "f"(v.z), "f"(v.w) : "memory");
}

// Dynamic shared memory: s_ids [256][K|1] int32, s_w [256][K|1] float.
template <int DT, int VPL, int G>
__global__ void __launch_bounds__(T)
batch_kernel(const BatchView *__restrict__ views, int n_views, uint32_t total_items,
             uint32_t *__restrict__ counter) {
    constexpr int CPV = VecT<DT>::C;
    constexpr int ROWV = 32 * VPL;
    constexpr unsigned FULL = 0xffffffffu;
    __shared__ float4 s_m[T];
    __shared__ float4 s_c[T];
    __shared__ float s_a[T];
    __shared__ float s_h[T];
    __shared__ uint32_t s_g[T];
    __shared__ uint32_t s_item;
    __shared__ uint8_t s_cnt[T];
    __shared__ __align__(16) float s_tw[T / 32][32][G];   // per-warp row-weight table
    __shared__ int s_tid[T / 32][32];
    extern __shared__ unsigned char s_dyn[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;

    for (;;) {
        if (threadIdx.x == 0) s_item = atomicAdd(counter, 1u);
        __syncthreads();
        const uint32_t item = s_item;
        __syncthreads();
        if (item >= total_items) break;
        int v = 0;
        for (int lo = 0, hi = n_views; hi - lo > 1;) {      // last view with tile_base <= item
            const int mid = (lo + hi) >> 1;
            if (views[mid].tile_base <= item) lo = mid; else hi = mid;
            v = lo;
        }
        const BatchView &V = views[v];
        const int K = V.K;
        const int KS = K | 1;   // odd stride: per-pixel slots fall in distinct banks
        int32_t *s_ids = reinterpret_cast<int32_t *>(s_dyn);          // [256][KS]
        float *s_w = reinterpret_cast<float *>(s_dyn) + KS * T;       // [256][KS]
        const int tile = int(item - V.tile_base);
        const int tx = tile % V.tiles_x, ty = tile / V.tiles_x;
        const int tile_w = V.tile_w, tile_h = T / tile_w;

        // ---------------- 1. selection (thread per pixel)
        {
            constexpr unsigned FULL = 0xffffffffu;
            const int lane = threadIdx.x & 31;
            const int lx = int(threadIdx.x) % tile_w, ly = int(threadIdx.x) / tile_w;
            const int px = tx * tile_w + lx, py = ty * tile_h + ly;
            const bool inside = px < V.W && py < V.H;
            const float ux = float(px) + 0.5f, uy = float(py) + 0.5f;
            const uint2 range = V.ranges[tile];
            const float tau_stop = __fdiv_rn(1.0f, float(K + 1));
            Walk wk{1.0f, 1.0f, __fdiv_rn(float(K), float(K + 1)), 0, 0, !inside};
            // the warp's box of pixel centres
            float bx0 = ux, bx1 = ux, by0 = uy, by1 = uy;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                bx0 = fminf(bx0, __shfl_xor_sync(FULL, bx0, o));
                bx1 = fmaxf(bx1, __shfl_xor_sync(FULL, bx1, o));
                by0 = fminf(by0, __shfl_xor_sync(FULL, by0, o));
                by1 = fmaxf(by1, __shfl_xor_sync(FULL, by1, o));
            }
            uint32_t gnext = range.x + threadIdx.x < range.y ? V.igid[range.x + threadIdx.x] : 0u;
            for (uint32_t b = range.x; b < range.y; b += T) {
                if (__syncthreads_count(wk.done) == T) break;
                if (b + threadIdx.x < range.y) {
                    s_g[threadIdx.x] = gnext;
                    s_m[threadIdx.x] = V.rec_m[gnext];
                    s_c[threadIdx.x] = V.rec_w[gnext];
                    s_a[threadIdx.x] = V.rec_a[gnext];
                    s_h[threadIdx.x] = V.rec_h[gnext];
                }
                __syncthreads();
                {
                    const uint32_t idx = b + T + threadIdx.x;
                    gnext = idx < range.y ? V.igid[idx] : 0u;
                }
                const int nb = int(min(uint32_t(T), range.y - b));
                for (int c0 = 0; c0 < nb; c0 += 32) {
                    if (__all_sync(FULL, wk.done)) break;
                    // per-warp culling against the box, as in qr_select
                    const int jl = c0 + lane;
                    bool pass = false;
                    if (jl < nb)
                        pass = !(box_min_half_q(s_m[jl], s_c[jl], bx0, bx1, by0, by1) * 0.999f > s_h[jl] + 1e-3f);
                    unsigned todo = __ballot_sync(FULL, pass);
                    while (todo) {
                        int jj[4];
                        bool valid[4];
#pragma unroll
                        for (int u = 0; u < 4; ++u) {
                            valid[u] = todo != 0u;
                            jj[u] = valid[u] ? c0 + __ffs(todo) - 1 : jj[0];
                            todo &= todo - 1u;
                        }
                        float hq[4];
                        unsigned reach = 0;
#pragma unroll
                        for (int u = 0; u < 4; ++u) {
                            hq[u] = eval_half_q(ux, uy, s_m[jj[u]], s_c[jj[u]]).half_q;
                            reach |= unsigned(valid[u] && !(hq[u] > s_h[jj[u]])) << u;
                        }
                        if (wk.done || !reach) continue;
#pragma unroll
                        for (int u = 0; u < 4; ++u) {
                            if (wk.done || !((reach >> u) & 1u)) continue;
                            const float a = eval_alpha(s_a[jj[u]], hq[u], V.alpha_max);
                            if (a < V.alpha_min) continue;
                            const float Tt = wk.T * (1.0f - a);
                            if (Tt < wk.thr || Tt < tau_stop)
                                walk_event(wk, Tt, a, tau_stop, K, s_g[jj[u]], threadIdx.x, KS, s_ids, s_w);
                            else
                                wk.T = Tt;
                        }
                        if (wk.done) break;
                    }
                }
            }
            // normalise this pixel's weights (Algorithm 1's 1 / (1 - T^Q)) in place
            const float D = 1.0f - wk.TQ;
            for (int j = 0; j < K; ++j) {
                const bool has = j < wk.m;
                s_w[threadIdx.x * KS + j] = has ? __fdiv_rn(s_w[threadIdx.x * KS + j], D) : 0.0f;
                if (!has) s_ids[threadIdx.x * KS + j] = -1;
            }
            s_cnt[threadIdx.x] = uint8_t(wk.m);
            __syncthreads();
            // coalesced output for a backward pass: each tile row is tile_w * K
            // consecutive ids and weights in the view
            const int rowlen = tile_w * K;
            for (int rem = threadIdx.x; rem < rowlen; rem += T) {
                const int cx = rem / K, j = rem - cx * K;
                const int gx = tx * tile_w + cx;
                if (gx >= V.W) continue;
                for (int row = 0; row < tile_h; ++row) {
                    const int gy = ty * tile_h + row;
                    if (gy >= V.H) break;
                    const int sl = row * tile_w + cx;
                    const int64_t o = (int64_t(gy) * V.W + gx) * K + j;
                    V.ids[o] = s_ids[sl * KS + j];
                    V.w[o] = s_w[sl * KS + j];
                }
            }
            if (inside) V.cnt[int64_t(py) * V.W + px] = s_cnt[threadIdx.x];
        }
        __syncthreads();

        // ---------------- 2. blend (warp per pixel group, rows shared in registers)
                const int half_w = tile_w / 2;
        for (int gi = warp; gi < T / G; gi += T / 32) {
            const int mm = lane / K, j = lane - mm * K;
            int lx, ly;
            if (G == 4) { lx = 2 * (gi % half_w) + (mm & 1); ly = 2 * (gi / half_w) + (mm >> 1); }
            else if (G == 2) { lx = 2 * (gi % half_w) + mm; ly = gi / half_w; }
            else { lx = gi % tile_w; ly = gi / tile_w; }
            const int loc = ly * tile_w + lx;
            const int px = tx * tile_w + lx, py = ty * tile_h + ly;
            int64_t p = -1;
            if (mm < G && px < V.W && py < V.H) p = int64_t(py) * V.W + px;
            int id = -1;
            float w = 0.f;
            if (p >= 0) {
                id = s_ids[loc * KS + j];
                w = s_w[loc * KS + j];
                if (id >= 0 && DT == QR_FP8E4M3) w *= V.fscale[id];
            }
            const unsigned peers = __match_any_sync(FULL, id);
            const int leader = __ffs(peers) - 1;
            const unsigned leaders = __ballot_sync(FULL, id >= 0 && lane == leader);
            const int nrows = __popc(leaders);
            // the G weights of each distinct row, gathered once (a pixel that
            // lists an id twice gets the sum)
#pragma unroll
            for (int g = 0; g < G; ++g) s_tw[warp][lane][g] = 0.f;
            __syncwarp();
            if (id >= 0) {
                const int slot = __popc(leaders & ((1u << leader) - 1u));
                atomicAdd(&s_tw[warp][slot][mm], w);
                if (lane == leader) s_tid[warp][slot] = id;
            }
            __syncwarp();
            float acc[G][VPL][CPV];
#pragma unroll
            for (int g = 0; g < G; ++g)
#pragma unroll
                for (int vv = 0; vv < VPL; ++vv)
#pragma unroll
                    for (int q = 0; q < CPV; ++q) acc[g][vv][q] = 0.f;
            const uint4 *feat = reinterpret_cast<const uint4 *>(V.feat);
            for (int r0 = 0; r0 < nrows; r0 += 2) {
                uint4 r[2][VPL];
#pragma unroll
                for (int u = 0; u < 2; ++u) {
                    const bool ok = r0 + u < nrows;
                    const uint4 *row = feat + int64_t(ok ? s_tid[warp][r0 + u] : 0) * ROWV + lane;
#pragma unroll
                    for (int vv = 0; vv < VPL; ++vv)
                        r[u][vv] = ok ? ldg_nc(row + 32 * vv) : make_uint4(0, 0, 0, 0);
                }
#pragma unroll
                for (int u = 0; u < 2; ++u) {
                    if (r0 + u >= nrows) break;
                    float wg[G];
#pragma unroll
                    for (int g = 0; g < G; ++g) wg[g] = s_tw[warp][r0 + u][g];
                    float fv[VPL][CPV];
#pragma unroll
                    for (int vv = 0; vv < VPL; ++vv) dec_vec<DT>(r[u][vv], fv[vv]);
#pragma unroll
                    for (int g = 0; g < G; ++g)
                        if (wg[g] != 0.f) {
#pragma unroll
                            for (int vv = 0; vv < VPL; ++vv)
#pragma unroll
                                for (int q = 0; q < CPV; q += 2)
                                    fma2b(acc[g][vv] + q, wg[g], fv[vv][q], fv[vv][q + 1]);
                        }
                }
            }
#pragma unroll
            for (int g = 0; g < G; ++g) {
                const int64_t pg = __shfl_sync(FULL, p, g * K < 32 ? g * K : 0);
                if (pg >= 0) {
                    float4 *o = reinterpret_cast<float4 *>(V.out) + pg * (int64_t(ROWV) * CPV / 4);
#pragma unroll
                    for (int vv = 0; vv < VPL; ++vv)
#pragma unroll
                        for (int q = 0; q < CPV / 4; ++q)
                            st_cs(o + int64_t(lane + 32 * vv) * (CPV / 4) + q,
                                  make_float4(acc[g][vv][4 * q], acc[g][vv][4 * q + 1],
                                              acc[g][vv][4 * q + 2], acc[g][vv][4 * q + 3]));
                }
            }
            __syncwarp();   // the table is rewritten by the next group
        }
        __syncthreads();
    }
}

template <int DT, int VPL, int G>
cudaError_t run_batch(const BatchView *dviews, int n_views, uint32_t total, uint32_t *counter,
                      int K, int ctas_per_sm, cudaStream_t s) {
    const size_t dyn = size_t(K | 1) * T * 8;
    cudaError_t e = cudaFuncSetAttribute(batch_kernel<DT, VPL, G>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, int(dyn));
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    int occ = 1;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, batch_kernel<DT, VPL, G>, T, dyn);
    if (ctas_per_sm > 0 && ctas_per_sm < occ) occ = ctas_per_sm;
    if (occ < 1) occ = 1;
    const uint32_t grid = uint32_t(sms) * uint32_t(occ);
    batch_kernel<DT, VPL, G><<<grid < total ? grid : total, T, dyn, s>>>(dviews, n_views, total, counter);
    count_launch();
    return cudaGetLastError();
}

template <int DT, int VPL>
cudaError_t pick_g(const BatchView *d, int n, uint32_t total, uint32_t *counter, int K, int group,
                   int ctas, cudaStream_t s) {
    const int g = group > 0 ? group : (K <= 8 ? 4 : K <= 16 ? 2 : 1);
    if (g == 4 && K <= 8) return run_batch<DT, VPL, 4>(d, n, total, counter, K, ctas, s);
    if (g >= 2 && K <= 16) return run_batch<DT, VPL, 2>(d, n, total, counter, K, ctas, s);
    return run_batch<DT, VPL, 1>(d, n, total, counter, K, ctas, s);
}

}  // namespace

bool batch_supported(qr_dtype dt, int C) {
    const int cpv = dt == QR_F32 ? 4 : dt == QR_BF16 ? 8 : 16;
    if (C <= 0 || C % cpv) return false;
    const int rowv = C / cpv;
    return rowv == 32 || rowv == 64 || rowv == 128;
}

size_t batch_desc_bytes(int n_views) { return (size_t(n_views) * sizeof(BatchView) + 255) / 256 * 256 + 256; }

cudaError_t launch_batch(const void *ws, int n_views, uint32_t total_items, qr_dtype dt, int C,
                         int K, int group, int ctas_per_sm, cudaStream_t s) {
    const BatchView *d = static_cast<const BatchView *>(ws);
    uint32_t *counter = reinterpret_cast<uint32_t *>(static_cast<char *>(const_cast<void *>(ws)) +
                                                     batch_desc_bytes(n_views) - 256);
    cudaError_t e = cudaMemsetAsync(counter, 0, 4, s);
    if (e != cudaSuccess) return e;
    const int rowv = C / (dt == QR_F32 ? 4 : dt == QR_BF16 ? 8 : 16);
    const int vpl = rowv / 32;
    switch (dt) {
        case QR_F32:
            if (vpl == 4) return pick_g<QR_F32, 4>(d, n_views, total_items, counter, K, group, ctas_per_sm, s);
            if (vpl == 2) return pick_g<QR_F32, 2>(d, n_views, total_items, counter, K, group, ctas_per_sm, s);
            return pick_g<QR_F32, 1>(d, n_views, total_items, counter, K, group, ctas_per_sm, s);
        case QR_BF16:
            if (vpl == 4) return pick_g<QR_BF16, 4>(d, n_views, total_items, counter, K, group, ctas_per_sm, s);
            if (vpl == 2) return pick_g<QR_BF16, 2>(d, n_views, total_items, counter, K, group, ctas_per_sm, s);
            return pick_g<QR_BF16, 1>(d, n_views, total_items, counter, K, group, ctas_per_sm, s);
        case QR_FP8E4M3:
            if (vpl == 4) return pick_g<QR_FP8E4M3, 4>(d, n_views, total_items, counter, K, group, ctas_per_sm, s);
            if (vpl == 2) return pick_g<QR_FP8E4M3, 2>(d, n_views, total_items, counter, K, group, ctas_per_sm, s);
            return pick_g<QR_FP8E4M3, 1>(d, n_views, total_items, counter, K, group, ctas_per_sm, s);
    }
    return cudaErrorInvalidValue;
}

// Host side of qr_batch_prepare: build the descriptors and copy them to ws.
cudaError_t prepare_batch(const qr_view *views, int n_views, void *ws, uint32_t *total_items,
                          cudaStream_t s, BatchView *host_scratch) {
    uint32_t base = 0;
    for (int i = 0; i < n_views; ++i) {
        const qr_frame &f = *views[i].frame;
        BatchView &b = host_scratch[i];
        b.rec_m = slot<float4>(f, S_REC_M);
        b.rec_w = slot<float4>(f, S_REC_C);
        b.rec_a = slot<float>(f, S_REC_A);
        b.rec_h = slot<float>(f, S_REC_H);
        b.igid = slot<uint32_t>(f, S_IGID);
        b.ranges = slot<uint2>(f, S_RANGES);
        b.feat = static_cast<const unsigned char *>(views[i].feat);
        b.fscale = views[i].feat_scale;
        b.ids = views[i].ids;
        b.w = views[i].weights;
        b.cnt = views[i].counts;
        b.out = views[i].out;
        b.n_gauss = f.n;
        b.W = f.camera.width;
        b.H = f.camera.height;
        b.tile_w = f.params.tile_w;
        b.tiles_x = f.tiles_x;
        b.tiles_y = f.tiles_y;
        b.K = f.params.K;
        b.alpha_min = f.params.alpha_min;
        b.alpha_max = f.params.alpha_max;
        b.tile_base = base;
        b.pad = 0;
        base += uint32_t(f.tiles_x * f.tiles_y);
    }
    *total_items = base;
    return cudaMemcpyAsync(ws, host_scratch, sizeof(BatchView) * size_t(n_views),
                           cudaMemcpyHostToDevice, s);
}

size_t batch_view_size() { return sizeof(BatchView); }

}  // namespace qr
