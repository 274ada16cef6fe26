// Many views in one persistent launch: Algorithm 1's selection and blend fused
// per screen tile, over the tiles of every view of a batch (the paper renders
// 4 random training views per scene per step, Appendix D; inference renders
// many views of several scenes).
//
// GB300 design: a grid of (SMs x resident CTAs) persistent CTAs pulls
// (view, tile) work items from one atomic counter, so views of very different
// sizes balance without a host round trip.  Each CTA is warp-specialised and
// double-buffered, so the latency-bound selection of one tile overlaps the
// bandwidth-bound blend of the previous one:
//   1. selection (warps 0-3, select_tile.cuh, the same code as qr_select):
//      the tile's depth-ordered list is staged through shared memory, culled
//      per warp against the warp's box of pixel centres and walked two pixels
//      per thread; the kept ids and normalised weights go to one of two
//      shared-memory buffers and are also written out (coalesced tile-row
//      runs) for a backward pass;
//   2. blend (8 warps, warp per 2x2 / 2x1 pixel group and channel chunk, like
//      qr_blend): equal ids of the group are merged with __match_any_sync, the
//      group's weights of each distinct row are gathered into a per-warp
//      table, each distinct feature row (or its chunk) is read once with
//      16-byte loads and accumulated into every pixel of the group, and the
//      rows of the map are written with streaming stores.
// Hand-over between the roles uses named barriers (below).  Per-view
// descriptors live in device memory (qr_batch_prepare), the counter is
// cleared by a memset on the stream, so the launch can sit in a CUDA graph.
#include <type_traits>

#include <cuda_bf16.h>
#include <cuda_fp8.h>

#include "quad.cuh"
#include "select_tile.cuh"

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

// ------------------------------------------------------------------ the kernel
// Warp roles of a CTA: warps 0..3 select (select_tile, 128 threads, two pixels
// each), warps 4..4+nbw-1 blend (nbw = 4 or 8, from the launch's block size).  Two shared-memory buffers hold a tile's
// kept ids, normalised weights and counts; the selection fills one while the
// blend warps read the other.  Hand-over uses hardware named barriers:
//   FULL[b]  (ids 2, 3): selection arrives once buffer b holds tile n (or the
//                        end marker), blend warps wait;
//   EMPTY[b] (ids 4, 5): blend warps arrive once done with buffer b, the
//                        selection waits before refilling it (from its third
//                        tile on) and once more after the end marker for the
//                        last tile's arrival, so every arrival is matched;
//   id 1:                the selection threads among themselves.
// Every thread of both roles runs the same number of barrier phases on each
// id, so no phase is left open and no wait can be missed.
constexpr int kNBW = 8;                               // blend warps at most
constexpr int kBT = kSelThreads + 32 * kNBW;          // threads per CTA at most
constexpr int kItemEnd = -1;

// Barrier ids are immediates (2 + b or 4 + b picked by a branch on b), so
// the kernel uses barriers 0..5 only; nt = the CTA's thread count.
template <int ID>
__device__ __forceinline__ void bar_sync_id(int nt) {
    asm volatile("bar.sync %0, %1;" ::"n"(ID), "r"(nt) : "memory");
}
template <int ID>
__device__ __forceinline__ void bar_arrive_id(int nt) {
    asm volatile("bar.arrive %0, %1;" ::"n"(ID), "r"(nt) : "memory");
}
__device__ __forceinline__ void full_sync(int b, int nt) { if (b) bar_sync_id<3>(nt); else bar_sync_id<2>(nt); }
__device__ __forceinline__ void full_arrive(int b, int nt) { if (b) bar_arrive_id<3>(nt); else bar_arrive_id<2>(nt); }
__device__ __forceinline__ void empty_sync(int b, int nt) { if (b) bar_sync_id<5>(nt); else bar_sync_id<4>(nt); }
__device__ __forceinline__ void empty_arrive(int b, int nt) { if (b) bar_arrive_id<5>(nt); else bar_arrive_id<4>(nt); }

__device__ __forceinline__ int find_view(const BatchView *views, int n_views, uint32_t item) {
    int lo = 0, hi = n_views;   // last view with tile_base <= item
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (views[mid].tile_base <= item) lo = mid; else hi = mid;
    }
    return lo;
}

// Dynamic shared memory: ids [2][256][KSB] int32, weights [2][256][KSB] float.
// QPL quads (4 channels) per lane per channel chunk, NCH chunks per row.
template <int DT, int QPL, int G, int NCH>
__global__ void __launch_bounds__(kBT, DT == QR_FP8E4M3 ? 1 : 2)
batch_kernel(const BatchView *__restrict__ views, int n_views, uint32_t total_items,
             uint32_t *__restrict__ counter, int KSB) {
    __shared__ SelStage st;
    __shared__ float s_D[kSelPix];
    __shared__ uint8_t s_cnt[2][kSelPix];
    __shared__ int s_item[2];
    __shared__ __align__(16) float s_tw[kNBW][32][G];   // per blend warp: row-weight table
    __shared__ int s_tid[kNBW][32];
    extern __shared__ __align__(16) unsigned char s_dyn[];
    int32_t *s_ids0 = reinterpret_cast<int32_t *>(s_dyn);
    float *s_w0 = reinterpret_cast<float *>(s_dyn) + 2 * kSelPix * KSB;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nt = int(blockDim.x), nbw = nt / 32 - kSelThreads / 32;

    if (warp < kSelThreads / 32) {
        // ------------------------------------------------ selection role
        using Bar = NamedBarrier<1, kSelThreads>;
        for (int n = 0;; ++n) {
            const int b = n & 1;
            if (n >= 2) empty_sync(b, nt);   // the blend warps are done with buffer b
            if (threadIdx.x == 0) {
                const uint32_t it = atomicAdd(counter, 1u);
                s_item[b] = it < total_items ? int(it) : kItemEnd;
            }
            Bar::sync();
            const int item = s_item[b];
            if (item == kItemEnd) {
                full_arrive(b, nt);
                if (n >= 1) empty_sync(b ^ 1, nt);   // the last tile's arrival
                break;
            }
            const BatchView &V = views[find_view(views, n_views, uint32_t(item))];
            const int K = V.K;
            int32_t *s_ids = s_ids0 + b * kSelPix * KSB;
            float *s_w = s_w0 + b * kSelPix * KSB;
            const int tile = item - int(V.tile_base);
            const int tx = tile % V.tiles_x, ty = tile / V.tiles_x;
            const int tile_w = V.tile_w, tile_h = kSelPix / tile_w;
            select_tile<Bar>(V.rec_m, V.rec_w, V.rec_a, V.rec_h, V.igid, V.ranges[tile], V.W, V.H,
                             tile_w, tx, ty, K, V.alpha_min, V.alpha_max, st, s_ids, s_w, s_D,
                             s_cnt[b]);
            // normalise this thread's two pixels in place (Algorithm 1's 1 / (1 - T^Q))
            {
                const int lx = threadIdx.x % tile_w, ly = 2 * (threadIdx.x / tile_w);
#pragma unroll
                for (int r = 0; r < 2; ++r) {
                    const int sl = (ly + r) * tile_w + lx;
                    const int c = s_cnt[b][sl];
                    const float D = s_D[sl];
                    for (int j = 0; j < K; ++j) {
                        const bool has = j < c;
                        s_w[sl * KSB + j] = has ? __fdiv_rn(s_w[sl * KSB + j], D) : 0.0f;
                        if (!has) s_ids[sl * KSB + j] = -1;
                    }
                }
            }
            Bar::sync();
            // coalesced output for a backward pass: each tile row is tile_w * K
            // consecutive ids and weights in the view
            const int rowlen = tile_w * K;
            for (int rem = threadIdx.x; rem < rowlen; rem += kSelThreads) {
                const int cx = rem / K, j = rem - cx * K;
                const int gx = tx * tile_w + cx;
                if (gx >= V.W) continue;
                for (int row = 0; row < tile_h; ++row) {
                    const int gy = ty * tile_h + row;
                    if (gy >= V.H) break;
                    const int sl = row * tile_w + cx;
                    const int64_t o = (int64_t(gy) * V.W + gx) * K + j;
                    V.ids[o] = s_ids[sl * KSB + j];
                    V.w[o] = s_w[sl * KSB + j];
                }
            }
            for (int e = threadIdx.x; e < kSelPix; e += kSelThreads) {
                const int gx = tx * tile_w + e % tile_w, gy = ty * tile_h + e / tile_w;
                if (gx < V.W && gy < V.H) V.cnt[int64_t(gy) * V.W + gx] = s_cnt[b][e];
            }
            full_arrive(b, nt);
        }
        return;
    }
    // ---------------------------------------------------- blend role
    constexpr int QB = Quad<DT>::B;
    constexpr int CQ = 32 * QPL;                 // quads of a channel chunk
    constexpr int ROWQ = CQ * NCH;               // quads of a row (C / 4)
    constexpr int U = QPL * QB >= 32 ? 2 : 4;    // rows in flight
    constexpr unsigned FULL = 0xffffffffu;
    constexpr int NITEMS = (kSelPix / G) * NCH;
    const int bw = warp - kSelThreads / 32;
    for (int n = 0;; ++n) {
        const int b = n & 1;
        full_sync(b, nt);   // buffer b holds a selected tile (or the end marker)
        const int item = s_item[b];
        if (item == kItemEnd) break;
        const BatchView &V = views[find_view(views, n_views, uint32_t(item))];
        const int K = V.K;
        const int32_t *s_ids = s_ids0 + b * kSelPix * KSB;
        const float *s_w = s_w0 + b * kSelPix * KSB;
        const int tile = item - int(V.tile_base);
        const int tx = tile % V.tiles_x, ty = tile / V.tiles_x;
        const int tile_w = V.tile_w, tile_h = kSelPix / tile_w;
        const int half_w = tile_w / 2;
        const unsigned char *feat = V.feat;
        const int mm = lane / K, j = lane - mm * K;
        for (int it = bw; it < NITEMS; it += nbw) {
            const int gi = it / NCH, ch = it - gi * NCH;
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
                id = s_ids[loc * KSB + j];
                w = s_w[loc * KSB + j];
            }
            const unsigned peers = __match_any_sync(FULL, id);
            const int leader = __ffs(peers) - 1;
            const unsigned leaders = __ballot_sync(FULL, id >= 0 && lane == leader);
            const int nrows = __popc(leaders);
            // the G weights of each distinct row, gathered once (a pixel that
            // lists an id twice gets the sum)
#pragma unroll
            for (int g = 0; g < G; ++g) s_tw[bw][lane][g] = 0.f;
            __syncwarp();
            if (id >= 0) {
                const int slot = __popc(leaders & ((1u << leader) - 1u));
                atomicAdd(&s_tw[bw][slot][mm], w);
                if (lane == leader) s_tid[bw][slot] = id;
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
                    const int rid = ok ? s_tid[bw][r0 + u] : 0;
                    const unsigned char *row = fch + size_t(rid) * (size_t(ROWQ) * QB);
#pragma unroll
                    for (int v = 0; v < QPL; ++v)
                        r[u][v] = ok ? ld_quad<DT>(row + size_t(32 * v) * QB) : zero_quad<DT>();
                    if (DT == QR_FP8E4M3) sc[u] = ok ? V.fscale[rid] : 0.f;
                }
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    if (r0 + u >= nrows) break;
                    float wg[G];
#pragma unroll
                    for (int g = 0; g < G; ++g)
                        wg[g] = DT == QR_FP8E4M3 ? s_tw[bw][r0 + u][g] * sc[u] : s_tw[bw][r0 + u][g];
                    float fv[QPL][4];
#pragma unroll
                    for (int v = 0; v < QPL; ++v) dec_quad<DT>(r[u][v], fv[v]);
#pragma unroll
                    for (int g = 0; g < G; ++g)
                        if (wg[g] != 0.f) {
#pragma unroll
                            for (int v = 0; v < QPL; ++v) {
                                fma2b(acc[g][v] + 0, wg[g], fv[v][0], fv[v][1]);
                                fma2b(acc[g][v] + 2, wg[g], fv[v][2], fv[v][3]);
                            }
                        }
                }
            }
#pragma unroll
            for (int g = 0; g < G; ++g) {
                const int64_t pg = __shfl_sync(FULL, p, g * K < 32 ? g * K : 0);
                if (pg >= 0) {
                    float4 *o = reinterpret_cast<float4 *>(V.out) + pg * int64_t(ROWQ) + ch * CQ + lane;
#pragma unroll
                    for (int v = 0; v < QPL; ++v)
                        st_cs(o + 32 * v, make_float4(acc[g][v][0], acc[g][v][1], acc[g][v][2],
                                                      acc[g][v][3]));
                }
            }
            __syncwarp();   // the table is rewritten by the next item
        }
        empty_arrive(b, nt);   // buffer b may be refilled
    }
}

template <int DT, int QT, int G, int NCH>
cudaError_t run_batch(const BatchView *dviews, int n_views, uint32_t total, uint32_t *counter,
                      int K, int nbw, int ctas_per_sm, cudaStream_t s) {
    auto kern = batch_kernel<DT, QT / NCH, G, NCH>;
    const int KSB = K | 1;
    const int nt = kSelThreads + 32 * nbw;
    const size_t dyn = size_t(KSB) * kSelPix * 2 * 8;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(dyn));
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    int occ = 1;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, nt, dyn);
    if (ctas_per_sm > 0 && ctas_per_sm < occ) occ = ctas_per_sm;
    if (occ < 1) occ = 1;
    const uint32_t grid = uint32_t(sms) * uint32_t(occ);
    kern<<<grid < total ? grid : total, nt, dyn, s>>>(dviews, n_views, total, counter, KSB);
    count_launch();
    return cudaGetLastError();
}

// Channel chunks per row by default: at most 2 quads (8 accumulators) per
// pixel and lane, so the blend warps fit the register budget of two CTAs
// per SM.
template <int QT>
constexpr int batch_default_chunks() {
    return QT <= 2 ? 1 : QT / 2;
}

// QT = C / 128 quads per lane over the whole row (1 .. 16).  group picks the
// pixel-group size (0 = largest allowed by K), chunks the channel chunks per
// row for groups of 4 (0 = default; 1, 2, 4 where they divide QT and leave at
// most 4 quads per lane).
template <int DT, int QT>
cudaError_t pick(const BatchView *d, int n, uint32_t total, uint32_t *counter, int K, int group,
                 int chunks, int nbw, int ctas, cudaStream_t s) {
    constexpr int DEF = batch_default_chunks<QT>();
    const int g = group > 0 ? group : (K <= 8 ? 4 : K <= 16 ? 2 : 1);
    if (g == 4 && K <= 8) {
        const int c = chunks > 0 ? chunks : DEF;
        if constexpr (QT <= 4)
            if (c == 1) return run_batch<DT, QT, 4, 1>(d, n, total, counter, K, nbw, ctas, s);
        if constexpr (QT % 2 == 0 && QT <= 8)
            if (c == 2) return run_batch<DT, QT, 4, 2>(d, n, total, counter, K, nbw, ctas, s);
        if constexpr (QT % 4 == 0 && QT <= 16)
            if (c == 4) return run_batch<DT, QT, 4, 4>(d, n, total, counter, K, nbw, ctas, s);
        if (chunks > 0) return cudaErrorInvalidValue;
        return run_batch<DT, QT, 4, DEF>(d, n, total, counter, K, nbw, ctas, s);
    }
    if (g >= 2 && K <= 16) return run_batch<DT, QT, 2, DEF>(d, n, total, counter, K, nbw, ctas, s);
    return run_batch<DT, QT, 1, DEF>(d, n, total, counter, K, nbw, ctas, s);
}

}  // namespace

bool batch_supported(qr_dtype dt, int C) {
    const int cpv = dt == QR_F32 ? 4 : dt == QR_BF16 ? 8 : 16;
    if (C <= 0 || C % cpv) return false;
    const int rowv = C / cpv;
    return rowv == 32 || rowv == 64 || rowv == 128;
}

bool batch_chunks_ok(int C, int chunks) {
    const int qt = C / 128;
    return chunks == 0 || (qt % chunks == 0 && qt / chunks <= 4);
}

size_t batch_desc_bytes(int n_views) { return (size_t(n_views) * sizeof(BatchView) + 255) / 256 * 256 + 256; }

cudaError_t launch_batch(const void *ws, int n_views, uint32_t total_items, qr_dtype dt, int C,
                         int K, int group, int chunks, int blend_warps, int ctas_per_sm,
                         cudaStream_t s) {
    const int nbw = blend_warps > 0 ? blend_warps : kNBW;
    const BatchView *d = static_cast<const BatchView *>(ws);
    uint32_t *counter = reinterpret_cast<uint32_t *>(static_cast<char *>(const_cast<void *>(ws)) +
                                                     batch_desc_bytes(n_views) - 256);
    cudaError_t e = cudaMemsetAsync(counter, 0, 4, s);
    if (e != cudaSuccess) return e;
    const int qt = C / 128;   // quads per lane over the whole row
    auto by_qt = [&](auto dtc) -> cudaError_t {
        constexpr int DT = decltype(dtc)::value;
        switch (qt) {
            case 1: return pick<DT, 1>(d, n_views, total_items, counter, K, group, chunks, nbw, ctas_per_sm, s);
            case 2: return pick<DT, 2>(d, n_views, total_items, counter, K, group, chunks, nbw, ctas_per_sm, s);
            case 4: return pick<DT, 4>(d, n_views, total_items, counter, K, group, chunks, nbw, ctas_per_sm, s);
            case 8: return pick<DT, 8>(d, n_views, total_items, counter, K, group, chunks, nbw, ctas_per_sm, s);
            case 16: return pick<DT, 16>(d, n_views, total_items, counter, K, group, chunks, nbw, ctas_per_sm, s);
        }
        return cudaErrorInvalidValue;
    };
    switch (dt) {
        case QR_F32: return by_qt(std::integral_constant<int, QR_F32>());
        case QR_BF16: return by_qt(std::integral_constant<int, QR_BF16>());
        case QR_FP8E4M3: return by_qt(std::integral_constant<int, QR_FP8E4M3>());
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
