// K6: dense alpha compositing, Eq. 1 of the paper (V-Render, the plain method
// Q-Render is compared against):
//     out[p] = sum_i T_i alpha'_i f_i,   T_i = prod_{j<i} (1 - alpha'_j)
// over the pixel's whole depth-ordered list, with the same alpha' rules as the
// selection and a stop before the Gaussian whose test transmittance would
// fall below T_min.
//
// GB300 design: every pixel of a tile walks the same list, so the blend is a
// dense product W (pixels x batch) * F (batch x channels) per batch of 32
// list entries.  Rows of 128, 256 or 512 channels go to dense_sub_kernel
// (below: one CTA per 64-pixel sub-tile over all channels, warp-specialised
// walk and accumulation).  Other widths use dense_kernel, where one CTA owns
// a screen tile and a 16/32/64-channel slice:
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

// ------------------------------------------------------------------ sub-tile kernel
// One CTA renders a 64-pixel sub-tile of a screen tile (16x4, 8x8 or 32x2)
// over all C channels (C = 64 CH, CH = 2, 4 or 8), so each pixel's alpha' / T
// walk runs once.  The CTA is warp-specialised and double-buffered, so the
// serial walk of one batch of list entries overlaps the accumulation of the
// previous one:
//   producers (warps 16, 17: one thread per pixel), per batch of 32 entries:
//     1. cull the batch's records (loaded into registers while the previous
//        batch was walked) against the sub-tile's box of pixel centres (the
//        conservative test of the selection);
//     2. walk every pixel over the survivors in list order (the scalar FP32
//        recurrence of dense_kernel) and write w = T alpha' into W[slot];
//     3. list, in list order, the survivors with a nonzero weight anywhere in
//        the sub-tile (and their ids);
//   consumers (warps 0-15: warps 2g and 2g+1 own pixel group g, a 4x2 block
//   of 8 pixels): stage the kept entries' feature rows in shared memory
//   (FP32 rows by 16-byte cp.async, BF16 / FP8 rows widened), then per kept
//   entry 8 weights and CH features per thread, 8 CH FMAs; an entry whose 8
//   weights are all zero is skipped by the warp.
// Hand-over through hardware named barriers: FULL[slot] (producers arrive
// once the slot is written, consumers wait) and EMPTY[slot] (consumers arrive
// once the slot is read, producers wait before writing it again and, at the
// end, for every slot still unread), so every barrier phase is matched.  A
// slot whose kept count is -1 ends the consumers' loop.  Zero weights add
// nothing (fmaf(0, f, acc) == acc), so the result equals dense_kernel's.
// stats (nullable): [0] += blended (pixel, Gaussian) pairs, [1] += executed
// multiply-adds.
constexpr int S_CONS = 512;                  // consumer threads (16 warps)
constexpr int S_PROD = 64;                   // producer threads (2 warps, one per pixel)
constexpr int S_THREADS = S_CONS + S_PROD;
constexpr int S_PIX = 64;
constexpr int S_BATCH = 32;
// named barriers (0 is __syncthreads)
constexpr int kBarFull = 1;                  // + slot
constexpr int kBarEmpty = 3;                 // + slot
constexpr int kBarProd = 5;
constexpr int kBarCons = 6;

__device__ __forceinline__ void nbar_sync(int id, int n) {
    asm volatile("bar.sync %0, %1;" :: "r"(id), "r"(n) : "memory");
}
__device__ __forceinline__ void nbar_arrive(int id, int n) {
    asm volatile("bar.arrive %0, %1;" :: "r"(id), "r"(n) : "memory");
}
__device__ __forceinline__ void cp_async16(void *smem, const void *gmem) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;"
                 :: "r"(uint32_t(__cvta_generic_to_shared(smem))), "l"(gmem) : "memory");
}

template <int DT, int CH>
__global__ void __launch_bounds__(S_THREADS, 1)
dense_sub_kernel(const float4 *__restrict__ rec_m, const float4 *__restrict__ rec_w,
                 const float *__restrict__ rec_a, const float *__restrict__ rec_h,
                 const uint32_t *__restrict__ isect_gid, const uint2 *__restrict__ ranges,
                 const unsigned char *__restrict__ feat, const float *__restrict__ fscale, int C,
                 int W, int H, int tile_w, int tiles_x, float alpha_min, float alpha_max,
                 float T_min, float *__restrict__ out, float *__restrict__ T_final,
                 unsigned long long *__restrict__ stats) {
    constexpr int CPV = Cpv<DT>::v;
    constexpr int ESZ = DT == QR_F32 ? 4 : DT == QR_BF16 ? 2 : 1;
    constexpr unsigned FULL = 0xffffffffu;
    // producer state
    __shared__ float4 s_m[S_BATCH];
    __shared__ float4 s_c[S_BATCH];
    __shared__ float s_a[S_BATCH];
    __shared__ float s_h[S_BATCH];
    __shared__ uint32_t s_g[S_BATCH];
    __shared__ int s_surv[S_BATCH];          // survivor -> staged entry
    __shared__ int s_ns;
    __shared__ int s_done[2];
    __shared__ float s_box[4];
    // double-buffered hand-over
    __shared__ __align__(16) float s_W[2][S_BATCH][S_PIX];
    __shared__ int s_used[2][S_BATCH];       // kept -> survivor
    __shared__ uint32_t s_kg[2][S_BATCH];    // kept -> Gaussian id
    __shared__ int s_nu[2];                  // kept entries, -1 = end
    extern __shared__ __align__(16) float s_F[];     // [S_BATCH][C], the consumers' rows

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int tile = blockIdx.x >> 2, sub = blockIdx.x & 3;
    const int tx = tile % tiles_x, ty = tile / tiles_x;
    const int tile_h = 256 / tile_w, sub_h = S_PIX / tile_w;
    const int gx_n = tile_w / 4;                       // pixel groups across
    // pixel slot ps = 8 g + i  ->  (lx, ly) in the sub-tile
    auto slot_xy = [&](int ps, int &x, int &y) {       // groups of 4 x 2 pixels
        const int g = ps >> 3, i = ps & 7;
        x = tx * tile_w + (g % gx_n) * 4 + (i & 3);
        y = ty * tile_h + sub * sub_h + (g / gx_n) * 2 + (i >> 2);
    };
    const uint2 range = ranges[tile];
    const bool producer = tid >= S_CONS;
    if (tid >= S_CONS && tid < S_CONS + 32) {
        // the sub-tile's box of pixel centres (clipped to the image)
        float bx0 = 1e30f, bx1 = -1e30f, by0 = 1e30f, by1 = -1e30f;
        for (int ps = lane; ps < S_PIX; ps += 32) {
            int x, y;
            slot_xy(ps, x, y);
            const float cx = float(x) + 0.5f, cy = float(y) + 0.5f;
            bx0 = fminf(bx0, cx); bx1 = fmaxf(bx1, cx); by0 = fminf(by0, cy); by1 = fmaxf(by1, cy);
        }
        for (int o = 16; o > 0; o >>= 1) {
            bx0 = fminf(bx0, __shfl_xor_sync(FULL, bx0, o));
            bx1 = fmaxf(bx1, __shfl_xor_sync(FULL, bx1, o));
            by0 = fminf(by0, __shfl_xor_sync(FULL, by0, o));
            by1 = fmaxf(by1, __shfl_xor_sync(FULL, by1, o));
        }
        if (lane == 0) { s_box[0] = bx0; s_box[1] = bx1; s_box[2] = by0; s_box[3] = by1; }
    }
    __syncthreads();
    const size_t row_bytes = size_t(C) * ESZ;

    if (producer) {
        // ---------------------------------------------------------- producers
        const int pt = tid - S_CONS, pw = pt >> 5;     // pixel slot, producer warp
        int px, py;
        slot_xy(pt, px, py);
        const bool inside = px < W && py < H;
        const float ux = float(px) + 0.5f, uy = float(py) + 0.5f;
        float T = 1.0f;
        bool done = !inside;
        unsigned long long n_blend = 0;
        bool pending[2] = {false, false};
        int sl = 0;
        // producer warp 0 holds the next batch's records in registers: their
        // loads (the list ids, then the records) run while the current batch
        // is walked
        uint32_t n_gid = 0;
        float4 n_m = make_float4(0.f, 0.f, 0.f, 0.f), n_c = n_m;
        float n_a = 0.f, n_h = 0.f;
        auto prefetch = [&](uint32_t bb) {
            if (pw == 0 && bb < range.y && uint32_t(lane) < range.y - bb) {
                n_gid = isect_gid[bb + lane];
                n_m = rec_m[n_gid];
                n_c = rec_w[n_gid];
                n_a = rec_a[n_gid];
                n_h = rec_h[n_gid];
            }
        };
        prefetch(range.x);
        for (uint32_t b = range.x;; b += S_BATCH) {
            const unsigned dv = __ballot_sync(FULL, done);
            if (lane == 0) s_done[pw] = dv == FULL;
            nbar_sync(kBarProd, S_PROD);
            const bool all_done = s_done[0] && s_done[1];
            nbar_sync(kBarProd, S_PROD);               // s_done is read before it is rewritten
            if (b >= range.y || all_done) break;
            const int nb = int(min(uint32_t(S_BATCH), range.y - b));
            // 1. stage and cull (producer warp 0, one entry per lane)
            if (pw == 0) {
                bool pass = false;
                if (lane < nb) {
                    s_g[lane] = n_gid;
                    s_m[lane] = n_m;
                    s_c[lane] = n_c;
                    s_a[lane] = n_a;
                    s_h[lane] = n_h;
                    pass = !(box_min_half_q(n_m, n_c, s_box[0], s_box[1], s_box[2], s_box[3]) * 0.999f >
                             n_h + 1e-3f);
                }
                const unsigned bal = __ballot_sync(FULL, pass);
                if (pass) s_surv[__popc(bal & ((1u << lane) - 1u))] = lane;
                if (lane == 0) s_ns = __popc(bal);
                prefetch(b + S_BATCH);
            }
            if (pending[sl]) {                        // the consumers are done with this slot
                nbar_sync(kBarEmpty + sl, S_THREADS);
                pending[sl] = false;
            }
            nbar_sync(kBarProd, S_PROD);
            const int ns = s_ns;
            // 2. the walk: W[slot][survivor][pixel slot]
            float(*Wt)[S_PIX] = s_W[sl];
            for (int sv = 0; sv < ns; ++sv) {
                const int j = s_surv[sv];
                float w = 0.f;
                if (!done) {
                    const PixelTerm ptm = eval_half_q(ux, uy, s_m[j], s_c[j]);
                    const float a = ptm.half_q > s_h[j] ? 0.f : eval_alpha(s_a[j], ptm.half_q, alpha_max);
                    if (a >= alpha_min) {
                        const float Tt = T * (1.0f - a);
                        if (T_min > 0.f && Tt < T_min) {
                            done = true;
                        } else {
                            w = T * a;
                            T = Tt;
                            ++n_blend;
                        }
                    }
                }
                Wt[sv][pt] = w;
            }
            nbar_sync(kBarProd, S_PROD);
            // 3. survivors with a nonzero weight, in list order, and their ids
            // (producer warp 0)
            if (pw == 0) {
                bool used = false;
                if (lane < ns) {
                    const float4 *wr = reinterpret_cast<const float4 *>(Wt[lane]);
#pragma unroll
                    for (int q = 0; q < S_PIX / 4; ++q) {
                        const float4 t = wr[q];
                        used |= (t.x != 0.f) | (t.y != 0.f) | (t.z != 0.f) | (t.w != 0.f);
                    }
                }
                const unsigned bal = __ballot_sync(FULL, used);
                if (used) {
                    const int u = __popc(bal & ((1u << lane) - 1u));
                    s_used[sl][u] = lane;
                    s_kg[sl][u] = s_g[s_surv[lane]];
                }
                if (lane == 0) s_nu[sl] = __popc(bal);
            }
            nbar_arrive(kBarFull + sl, S_THREADS);
            pending[sl] = true;
            sl ^= 1;
        }
        // the end marker, then wait until every produced slot has been read
        if (pending[sl]) {
            nbar_sync(kBarEmpty + sl, S_THREADS);
            pending[sl] = false;
        }
        if (pt == 0) s_nu[sl] = -1;
        nbar_arrive(kBarFull + sl, S_THREADS);
        sl ^= 1;
        if (pending[sl]) nbar_sync(kBarEmpty + sl, S_THREADS);
        if (T_final && inside) T_final[int64_t(py) * W + px] = T;
        if (stats) atomicAdd(&stats[0], n_blend);
        return;
    }

    // -------------------------------------------------------------- consumers
    // thread t of a group's warp pair owns the channel pairs 2 t + 128 k
    // (k < CH / 2), so a warp's shared-memory reads and global writes are
    // consecutive 8-byte pairs
    const int g = warp >> 1;
    const int c0 = (tid & 63) * 2;
    float acc[8][CH];
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int c = 0; c < CH; ++c) acc[i][c] = 0.f;
    unsigned long long n_exec = 0;
    for (int sl = 0;; sl ^= 1) {
        nbar_sync(kBarFull + sl, S_THREADS);
        const int nu = s_nu[sl];
        if (nu < 0) break;
        // the kept rows into F (the consumers are all past the previous
        // batch: the FULL barrier counts every one of them)
        const int vpr = C / CPV;                       // 16-byte vectors per row
        for (int i = tid; i < nu * vpr; i += S_CONS) {
            const int u = i / vpr, v = i - u * vpr;
            const uint32_t gid = s_kg[sl][u];
            const unsigned char *src = feat + size_t(gid) * row_bytes + size_t(v) * 16;
            if constexpr (DT == QR_F32) {
                cp_async16(s_F + size_t(u) * C + v * CPV, src);
            } else {
                const uint4 x = __ldg(reinterpret_cast<const uint4 *>(src));
                float tmp[CPV];
                widen16<DT>(x, DT == QR_FP8E4M3 ? fscale[gid] : 1.f, tmp);
#pragma unroll
                for (int q = 0; q < CPV; q += 4)
                    *reinterpret_cast<float4 *>(s_F + size_t(u) * C + v * CPV + q) =
                        make_float4(tmp[q], tmp[q + 1], tmp[q + 2], tmp[q + 3]);
            }
        }
        if constexpr (DT == QR_F32) asm volatile("cp.async.wait_all;" ::: "memory");
        nbar_sync(kBarCons, S_CONS);
        for (int u = 0; u < nu; ++u) {
            const int sv = s_used[sl][u];
            const float4 *wr = reinterpret_cast<const float4 *>(&s_W[sl][sv][g * 8]);
            const float4 wa = wr[0], wb = wr[1];
            const float wv[8] = {wa.x, wa.y, wa.z, wa.w, wb.x, wb.y, wb.z, wb.w};
            const bool any = (wa.x != 0.f) | (wa.y != 0.f) | (wa.z != 0.f) | (wa.w != 0.f) |
                             (wb.x != 0.f) | (wb.y != 0.f) | (wb.z != 0.f) | (wb.w != 0.f);
            if (!any) continue;
            ++n_exec;
            const float *Fr = s_F + size_t(u) * C;
            float fv[CH];
#pragma unroll
            for (int k = 0; k < CH / 2; ++k) {
                const float2 t = *reinterpret_cast<const float2 *>(Fr + 128 * k + c0);
                fv[2 * k] = t.x;
                fv[2 * k + 1] = t.y;
            }
#pragma unroll
            for (int i = 0; i < 8; ++i)
#pragma unroll
                for (int c = 0; c < CH; ++c) acc[i][c] = fmaf(wv[i], fv[c], acc[i][c]);
        }
        nbar_arrive(kBarEmpty + sl, S_THREADS);
    }
    // write the sub-tile
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        int x, y;
        slot_xy(g * 8 + i, x, y);
        if (x < W && y < H) {
            float *o = out + (int64_t(y) * W + x) * C + c0;
#pragma unroll
            for (int k = 0; k < CH / 2; ++k)
                *reinterpret_cast<float2 *>(o + 128 * k) = make_float2(acc[i][2 * k], acc[i][2 * k + 1]);
        }
    }
    // executed FMAs (a warp's entries x 32 lanes x 8 pixels x CH)
    if (stats && lane == 0) atomicAdd(&stats[1], n_exec * 32ull * 8ull * CH);
}

template <int DT, int CH>
cudaError_t run_sub(const qr_frame &f, const void *feat, const float *scale, int C, float *out,
                    float *T_final, unsigned long long *stats, cudaStream_t s) {
    const size_t dyn = size_t(S_BATCH) * C * 4;
    cudaError_t e = cudaFuncSetAttribute(dense_sub_kernel<DT, CH>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, int(dyn));
    if (e != cudaSuccess) return e;
    dense_sub_kernel<DT, CH><<<unsigned(num_tiles(f)) * 4, S_THREADS, dyn, s>>>(
        slot<float4>(f, S_REC_M), slot<float4>(f, S_REC_C), slot<float>(f, S_REC_A),
        slot<float>(f, S_REC_H), slot<uint32_t>(f, S_IGID), slot<uint2>(f, S_RANGES),
        static_cast<const unsigned char *>(feat), scale, C, f.camera.width, f.camera.height,
        f.params.tile_w, f.tiles_x, f.params.alpha_min, f.params.alpha_max, f.params.T_min, out,
        T_final, stats);
    count_launch();
    return cudaGetLastError();
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
                     float *T_final, unsigned long long *stats, cudaStream_t s) {
    constexpr int cpv = Cpv<DT>::v;
    // wide rows: the sub-tile kernel (one walk per pixel, culled and skipped entries)
    if (C == 512) return run_sub<DT, 8>(f, feat, scale, C, out, T_final, stats, s);
    if (C == 256) return run_sub<DT, 4>(f, feat, scale, C, out, T_final, stats, s);
    if (C == 128 && cpv <= 8) return run_sub<DT, 2>(f, feat, scale, C, out, T_final, stats, s);
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
                         int C, float *out, float *T_final, cudaStream_t s,
                         unsigned long long *stats) {
    if (num_tiles(f) == 0) return cudaSuccess;
    switch (dt) {
        case QR_F32: return dispatch<QR_F32>(f, feat, scale, C, out, T_final, stats, s);
        case QR_BF16: return dispatch<QR_BF16>(f, feat, scale, C, out, T_final, stats, s);
        case QR_FP8E4M3: return dispatch<QR_FP8E4M3>(f, feat, scale, C, out, T_final, stats, s);
    }
    return cudaErrorInvalidValue;
}

}  // namespace qr
