// K7: backward of Algorithm 1 (Sec. 4.2).  The paper states that gradients of
// image-space losses flow through Q-Render into the per-Gaussian features
// (Sec. 1, Sec. 4.2) but prints no formula; this is the derivation the FP64
// oracle pins with finite differences.  For the quantile Gaussians j = 1..m of
// a pixel (depth order) with a_j = alpha'_j, P_j = prod_{l<j} (1 - a_l),
// T^Q = P_{m+1}, D = 1 - T^Q, F = sum_j a_j P_j f_j / D and g = dL/dF:
//   dL/df_j = w_j g                                   (w_j = a_j P_j / D)
//   dL/da_j = [P_j s_j - (1-a_j)^{-1} sum_{l>j} a_l P_l s_l] / D
//             - (g.F) T^Q / ((1-a_j) D),                s_l = g . f_l
//   dL/dalpha = dL/da G,  dL/d(A00,A01,A11) = dL/da (-a/2) (dx^2, 2 dx dy, dy^2)
// (zero where alpha G reached alpha_max).  The selection is held fixed.
//
// GB300 design -- deterministic, no floating-point atomics:
//   1. bwd_pixel: one warp per pixel recomputes its quantile Gaussians' alpha'
//      with the forward's exact evaluation, forms s_j with warp-wide dot
//      products (16-byte feature loads, BF16/FP8 decoded in registers) and
//      writes per-entry (dalpha, dA00, dA01, dA11); with the cosine loss
//      fused, it first forms the pixel's dL/dF itself;
//   2. bwd_tile_partials: one CTA per screen tile sorts the tile's (Gaussian,
//      entry) keys once (in registers), stages each entry's pixel and weight
//      and, 64 channels at a time, the tile's rows of g in shared memory, and
//      sums each distinct Gaussian's w * g rows in entry order into a partial
//      row, stored at a fixed slot of that tile's intersection range (slots
//      in ascending Gaussian id);
//   3. bwd_selected + bwd_rows: each Gaussian that survived the projection
//      owns a slot map (one entry per tile of its footprint rectangle, at its
//      intersection offset) that step 2 fills for the tiles that selected it;
//      the first tile to select a Gaussian lists it, and one CTA per listed
//      Gaussian (bwd_rows; 1024 threads for large footprints) adds its
//      partials in tile order (warps over channel blocks and fixed row
//      subsets).  Rows of unselected Gaussians stay as cleared.
#include <cstring>
#include <mutex>

#include <cuda_bf16.h>
#include <cuda_fp8.h>

#include "qr_internal.cuh"
#include "tma.cuh"

namespace qr {
namespace {

constexpr int T = 256;
constexpr int kRowsSmall = 64;    // selected Gaussians' maps up to this many tiles: 256-thread row CTAs

template <int DT> struct VecB;
template <> struct VecB<QR_F32> { static constexpr int C = 4; static constexpr int E = 4; };
template <> struct VecB<QR_BF16> { static constexpr int C = 8; static constexpr int E = 2; };
template <> struct VecB<QR_FP8E4M3> { static constexpr int C = 16; static constexpr int E = 1; };

template <int DT>
__device__ __forceinline__ void widen(const uint4 v, float *o);
template <>
__device__ __forceinline__ void widen<QR_F32>(const uint4 v, float *o) {
    o[0] = __uint_as_float(v.x); o[1] = __uint_as_float(v.y);
    o[2] = __uint_as_float(v.z); o[3] = __uint_as_float(v.w);
}
template <>
__device__ __forceinline__ void widen<QR_BF16>(const uint4 v, float *o) {
    const uint32_t u[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        o[2 * i] = __uint_as_float(u[i] << 16);
        o[2 * i + 1] = __uint_as_float(u[i] & 0xFFFF0000u);
    }
}
template <>
__device__ __forceinline__ void widen<QR_FP8E4M3>(const uint4 v, float *o) {
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

// ------------------------------------------------------------------ 1. per pixel
// LOSS: the upstream gradient is the cosine loss's, formed here from the map
// F and the target (the lane's slices, held in registers) and written to
// grad_out; the pixel's loss term goes to term.  Needs VPL > 0.
struct PixLoss {
    const float *F;
    const float *tgt;
    const uint8_t *mask;
    float *term;
    const float *out2;
};

// Four partial sums per lane reduced over the warp with 7 shuffles instead of
// 20: two halving levels (lane bits 4 and 3 pick which sums a lane keeps),
// then a plain butterfly over bits 2..0.  Lane l ends with the full sum of
// value 2 ((l >> 4) & 1) + ((l >> 3) & 1); red4_lane(u) is a lane holding u.
__device__ __forceinline__ float reduce4(float (&v)[4], int lane) {
    constexpr unsigned FULL = 0xffffffffu;
    const bool u16 = (lane & 16) != 0, u8 = (lane & 8) != 0;
    const float k0 = u16 ? v[2] : v[0], k1 = u16 ? v[3] : v[1];
    const float s0 = u16 ? v[0] : v[2], s1 = u16 ? v[1] : v[3];
    const float w0 = k0 + __shfl_xor_sync(FULL, s0, 16);
    const float w1 = k1 + __shfl_xor_sync(FULL, s1, 16);
    float x = (u8 ? w1 : w0) + __shfl_xor_sync(FULL, u8 ? w0 : w1, 8);
#pragma unroll
    for (int o = 4; o > 0; o >>= 1) x += __shfl_xor_sync(FULL, x, o);
    return x;
}
__device__ __forceinline__ int red4_lane(int u) { return ((u >> 1) << 4) | ((u & 1) << 3); }

template <int DT, int VPL, bool LOSS>
__global__ void __launch_bounds__(T)
bwd_pixel(const float4 *__restrict__ rec_m, const float4 *__restrict__ rec_w,
          const float *__restrict__ rec_a, const unsigned char *__restrict__ feat,
          const float *__restrict__ fscale, int C, const int32_t *__restrict__ ids,
          const float *__restrict__ wts, const uint8_t *__restrict__ cnt,
          float *__restrict__ grad_out, int64_t P, int K, int W, float alpha_max,
          float4 *__restrict__ E, PixLoss loss) {
    constexpr int CPV = VecB<DT>::C, ESZ = VecB<DT>::E;
    constexpr unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const int64_t warp0 = (int64_t(blockIdx.x) * T + threadIdx.x) >> 5;
    const int64_t nw = (int64_t(gridDim.x) * T) >> 5;
    const int nvec = C / CPV;                      // 16-byte vectors per feature row
    const size_t row_bytes = size_t(C) * ESZ;
    const float inv_n = LOSS ? cos_inv_count(loss.out2) : 0.f;
    for (int64_t p = warp0; p < P; p += nw) {
        const int m = cnt[p];
        // the pixel's entries, loaded before (and independently of) its rows
        const int id = lane < m ? ids[p * K + lane] : 0;
        const float wj = lane < m ? wts[p * K + lane] : 0.f;
        float gr[VPL > 0 ? VPL : 1][CPV];
        float *g = grad_out + p * int64_t(C);
        if (LOSS) {
            // the loss term and dL/dF of this pixel (every pixel, zero rows
            // outside the mask), as the loss's own pass computes them
            const bool on = loss.mask[p] > 0;
            float tr[VPL > 0 ? VPL : 1][CPV];
            float dot = 0.f, ff = 0.f, tt = 0.f;
#pragma unroll
            for (int t = 0; t < VPL; ++t) {
                const float4 *fv = reinterpret_cast<const float4 *>(loss.F + p * int64_t(C) + (lane + 32 * t) * CPV);
                const float4 *tv = reinterpret_cast<const float4 *>(loss.tgt + p * int64_t(C) + (lane + 32 * t) * CPV);
#pragma unroll
                for (int q = 0; q < CPV / 4; ++q) {
                    const float4 a = fv[q], b = tv[q];
                    gr[t][4 * q] = a.x; gr[t][4 * q + 1] = a.y; gr[t][4 * q + 2] = a.z; gr[t][4 * q + 3] = a.w;
                    tr[t][4 * q] = b.x; tr[t][4 * q + 1] = b.y; tr[t][4 * q + 2] = b.z; tr[t][4 * q + 3] = b.w;
                }
            }
#pragma unroll
            for (int t = 0; t < VPL; ++t)
#pragma unroll
                for (int q = 0; q < CPV; ++q) {
                    dot = fmaf(gr[t][q], tr[t][q], dot);
                    ff = fmaf(gr[t][q], gr[t][q], ff);
                    tt = fmaf(tr[t][q], tr[t][q], tt);
                }
            {
                float v4[4] = {dot, ff, tt, 0.f};
                const float x = reduce4(v4, lane);
                dot = __shfl_sync(FULL, x, red4_lane(0));
                ff = __shfl_sync(FULL, x, red4_lane(1));
                tt = __shfl_sync(FULL, x, red4_lane(2));
            }
            const CosCoeffs cc = cos_coeffs(dot, ff, tt, 1e-8f);
            if (lane == 0) loss.term[p] = on ? 1.f - cc.cs : 0.f;
#pragma unroll
            for (int t = 0; t < VPL; ++t) {
#pragma unroll
                for (int q = 0; q < CPV; ++q)
                    gr[t][q] = on ? -(tr[t][q] * cc.k1 - gr[t][q] * cc.k2) * inv_n : 0.f;
                float4 *gv = reinterpret_cast<float4 *>(g + (lane + 32 * t) * CPV);
#pragma unroll
                for (int q = 0; q < CPV / 4; ++q)
                    __stcg(gv + q, make_float4(gr[t][4 * q], gr[t][4 * q + 1], gr[t][4 * q + 2], gr[t][4 * q + 3]));
            }
        }
        if (m == 0) continue;
        const float ux = float(p % W) + 0.5f, uy = float(p / W) + 0.5f;
        // s_j = g . f_j for every quantile Gaussian j (lane j keeps s_j): the
        // lane's slice of g is held in registers, four rows are loaded at once
        // and their four partial dots reduced together
        float s_mine = 0.f;
        if (VPL > 0) {
            if (!LOSS) {
#pragma unroll
                for (int t = 0; t < VPL; ++t) {
                    const float4 *gv = reinterpret_cast<const float4 *>(g + (lane + 32 * t) * CPV);
#pragma unroll
                    for (int q = 0; q < CPV / 4; ++q) {
                        const float4 gg = gv[q];
                        gr[t][4 * q] = gg.x; gr[t][4 * q + 1] = gg.y; gr[t][4 * q + 2] = gg.z; gr[t][4 * q + 3] = gg.w;
                    }
                }
            }
            for (int j0 = 0; j0 < m; j0 += 4) {
                uint4 rv[4][VPL > 0 ? VPL : 1];
                float sc4[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int jj = j0 + u < m ? j0 + u : j0;
                    const int gj = __shfl_sync(FULL, id, jj);
                    const unsigned char *row = feat + size_t(gj) * row_bytes;
                    sc4[u] = (DT == QR_FP8E4M3) ? fscale[gj] : 1.f;
#pragma unroll
                    for (int t = 0; t < VPL; ++t)
                        rv[u][t] = *reinterpret_cast<const uint4 *>(row + size_t(lane + 32 * t) * 16);
                }
                float part[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    part[u] = 0.f;
#pragma unroll
                    for (int t = 0; t < VPL; ++t) {
                        float fv[CPV];
                        widen<DT>(rv[u][t], fv);
#pragma unroll
                        for (int q = 0; q < CPV; ++q) part[u] = fmaf(fv[q], gr[t][q], part[u]);
                    }
                }
                // lane j0 + u takes row u's dot from a lane that holds it
                const float x = reduce4(part, lane);
                const int u = lane - j0;
                const float su = __shfl_sync(FULL, x, red4_lane(u & 3));
                if (u >= 0 && u < 4 && lane < m) s_mine = su * sc4[u & 3];
            }
        } else {
            for (int j = 0; j < m; ++j) {
                const int gj = __shfl_sync(FULL, id, j);
                const unsigned char *row = feat + size_t(gj) * row_bytes;
                const float sc = (DT == QR_FP8E4M3) ? fscale[gj] : 1.f;
                float part = 0.f;
                for (int v = lane; v < nvec; v += 32) {
                    float fv[CPV];
                    widen<DT>(*reinterpret_cast<const uint4 *>(row + size_t(v) * 16), fv);
                    const float4 *gv = reinterpret_cast<const float4 *>(g + v * CPV);
#pragma unroll
                    for (int q = 0; q < CPV / 4; ++q) {
                        const float4 gg = gv[q];
                        part = fmaf(fv[4 * q], gg.x, part);
                        part = fmaf(fv[4 * q + 1], gg.y, part);
                        part = fmaf(fv[4 * q + 2], gg.z, part);
                        part = fmaf(fv[4 * q + 3], gg.w, part);
                    }
                }
                for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(FULL, part, o);
                if (lane == j) s_mine = part * sc;
            }
        }
        // alpha', G, offsets of this lane's Gaussian, recomputed exactly as in the forward
        float a = 0.f, G = 0.f, dx = 0.f, dy = 0.f;
        bool clamped = false;
        if (lane < m) {
            const PixelTerm t = eval_half_q(ux, uy, rec_m[id], rec_w[id]);
            const float alpha = rec_a[id];
            G = __expf(-t.half_q);
            a = eval_alpha(alpha, t.half_q, alpha_max);
            clamped = !(alpha * G < alpha_max);
            dx = t.dx;
            dy = t.dy;
        }
        // prefix products, T^Q, g.F and suffix sums (sequential, like the forward)
        float Pj = 1.f, Pmine = 1.f, gF = 0.f;
        for (int j = 0; j < m; ++j) {
            if (lane == j) Pmine = Pj;
            const float aj = __shfl_sync(FULL, a, j);
            gF = fmaf(__shfl_sync(FULL, wj, j), __shfl_sync(FULL, s_mine, j), gF);
            Pj = Pj * (1.f - aj);
        }
        const float TQ = Pj, D = 1.f - TQ;
        float suffix = 0.f, smine_suffix = 0.f;
        for (int j = m - 1; j >= 0; --j) {
            if (lane == j) smine_suffix = suffix;
            const float aj = __shfl_sync(FULL, a, j), pj = __shfl_sync(FULL, Pmine, j),
                        sj = __shfl_sync(FULL, s_mine, j);
            suffix = fmaf(aj * pj, sj, suffix);
        }
        if (lane < m) {
            const float om = 1.f - a;
            const float da = (Pmine * s_mine - smine_suffix / om) / D - gF * TQ / (om * D);
            float4 e = make_float4(0.f, 0.f, 0.f, 0.f);
            if (!clamped) {
                const float h = -0.5f * a * da;
                e = make_float4(da * G, h * dx * dx, h * 2.f * dx * dy, h * dy * dy);
            }
            E[p * K + lane] = e;
        }
    }
}

// acc += w * g for both halves with one packed FP32x2 FMA (each half rounds
// exactly like fmaf).
__device__ __forceinline__ void fma2v(float2 &acc, float w, float2 g) {
    asm("{\n .reg .b64 a, ww, xx;\n mov.b64 a, {%0, %1};\n mov.b64 ww, {%2, %2};\n"
        " mov.b64 xx, {%3, %4};\n fma.rn.f32x2 a, ww, xx, a;\n mov.b64 {%0, %1}, a;\n}\n"
        : "+f"(acc.x), "+f"(acc.y) : "f"(w), "f"(g.x), "f"(g.y));
}

// acc += w * g for four channels: two packed FP32x2 FMAs
__device__ __forceinline__ void fma4v(float4 &acc, float w, float4 g) {
    float2 lo = make_float2(acc.x, acc.y), hi = make_float2(acc.z, acc.w);
    fma2v(lo, w, make_float2(g.x, g.y));
    fma2v(hi, w, make_float2(g.z, g.w));
    acc = make_float4(lo.x, lo.y, hi.x, hi.y);
}

// ------------------------------------------------------------------ 2. per tile
__device__ __forceinline__ void bitonic64(unsigned long long *s, int npow2) {
    for (int k = 2; k <= npow2; k <<= 1)
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int i = threadIdx.x; i < npow2; i += T) {
                const int ixj = i ^ j;
                if (ixj > i) {
                    const unsigned long long x = s[i], y = s[ixj];
                    if ((x > y) == ((i & k) == 0)) { s[i] = y; s[ixj] = x; }
                }
            }
            __syncthreads();
        }
}

// One CTA per tile (256 threads, one per pixel).  The tile's (gid, pixel * K +
// entry) keys -- 32-bit (gid << 11 | local) when every gid is below 2^21 and
// K <= 8, else 64-bit (gid << 32 | local) -- are sorted once (E = 1..8 per
// thread in registers when K <= 8, else a shared-memory network), so the
// entries of each distinct Gaussian form a segment in (pixel, entry) order.
// Each entry's pixel and weight are then gathered into shared memory in
// sorted order with independent loads; the (dalpha, dA) terms are summed per
// segment by a warp's lanes in a fixed order.  Per CH-channel chunk, the
// tile's rows of g are staged in shared memory (by TMA when a tensor map is
// given, the next chunk's copy issued as soon as the walk has read the
// current one) and the warps walk equal shares of the entries (see below),
// each segment's w * g[pixel] sum going to its partial row at slot range.x +
// segment of the tile's intersection range.
constexpr unsigned kTmaSpin = 1u << 26;   // polls before a staging wait gives up

template <int E, typename KT>
__global__ void __launch_bounds__(T)
bwd_tile_partials(const uint2 *__restrict__ ranges, int W, int H, int tile_w, int tiles_x,
                  const int32_t *__restrict__ ids, const float *__restrict__ wts,
                  const uint8_t *__restrict__ cnt, const float4 *__restrict__ E4,
                  const float *__restrict__ grad_out, int C, int K, int CH,
                  float *__restrict__ partial, float4 *__restrict__ partial_s,
                  const uint2 *__restrict__ rect, const uint32_t *__restrict__ tcount,
                  const uint32_t *__restrict__ goff, uint32_t *__restrict__ slotmap, int64_t X,
                  uint32_t *__restrict__ gflag, uint32_t *__restrict__ lists, int64_t N,
                  const __grid_constant__ CUtensorMap gmap, int use_tma,
                  uint32_t *__restrict__ counters) {
    constexpr bool K32 = sizeof(KT) == 4;
    constexpr int SHIFT = K32 ? 11 : 32;
    extern __shared__ __align__(16) unsigned char s_dyn[];
    __shared__ uint32_t s_w[32];
    __shared__ uint32_t s_nseg;
    __shared__ __align__(8) uint64_t s_bar[1];
    __shared__ int s_ok;
    // per chunk parity, per warp: the continued and the begun piece (64 channels each)
    __shared__ __align__(16) float4 s_piece[2][(T / 32) * 2 * 16];
    __shared__ int s_first[2][T / 32], s_last[2][T / 32];
    int npow2 = 1;
    while (npow2 < T * K) npow2 <<= 1;
    // 1024-byte aligned base (the launch adds 1 KB of slack for it), formed as an
    // offset from the shared array so every access below stays a shared-memory
    // access (a round trip through an integer address would make them generic)
    unsigned char *base = s_dyn + ((1024u - (uint32_t(__cvta_generic_to_shared(s_dyn)) & 1023u)) & 1023u);
    KT *s_key = reinterpret_cast<KT *>(base);                                    // npow2
    uint32_t *seg = reinterpret_cast<uint32_t *>(s_key + npow2);                 // T*K
    uint2 *s_ent = reinterpret_cast<uint2 *>(seg + T * K);                       // T*K (pixel, w)
    const size_t g_off = (size_t(npow2) * sizeof(KT) + size_t(T * K) * 12 + 1023) & ~size_t(1023);
    float *s_g = reinterpret_cast<float *>(base + g_off);                       // [T*CH]
    const int tile = blockIdx.x;
    const int tx = tile % tiles_x, ty = tile / tiles_x;
    const int tile_h = T / tile_w;
    const int px = tx * tile_w + threadIdx.x % tile_w, py = ty * tile_h + threadIdx.x / tile_w;
    const bool inside = px < W && py < H;
    const int64_t p = inside ? int64_t(py) * W + px : 0;
    const uint2 r = ranges[tile];
    const int m = inside ? int(cnt[p]) : 0;
    uint32_t tot;
    block_inclusive_scan(uint32_t(m), s_w, tot);
    const int n = int(tot);
    if (n == 0) {
        return;
    }
    const int nchunks = (C + CH - 1) / CH;
    const uint32_t chunk_bytes = uint32_t(T) * uint32_t(CH) * 4u;
    if (use_tma && threadIdx.x == 0) {
        // the first chunk of g flies while the keys are sorted
        tma_mbar_init(&s_bar[0], 1);
        tma_fence_init();
        tma_expect_tx(&s_bar[0], chunk_bytes);
        tma_load_3d(s_g, &gmap, 0, tx * tile_w, ty * tile_h, &s_bar[0]);
    }
    auto key_of = [&](int j) -> KT {
        return j < m ? (KT(uint32_t(ids[p * K + j])) << SHIFT) | KT(uint32_t(threadIdx.x * K + j))
                     : ~KT(0);
    };
    if constexpr (E > 0) {
        KT v[E];
#pragma unroll
        for (int e = 0; e < E; ++e) v[e] = key_of(e);
        bitonic_regs<E, T, KT>(v, s_key);
        __syncthreads();
#pragma unroll
        for (int e = 0; e < E; ++e) s_key[threadIdx.x * E + e] = v[e];
    } else {
        for (int j = 0; j < K; ++j) s_key[threadIdx.x * K + j] = key_of(j);
        for (int i = T * K + threadIdx.x; i < npow2; i += T) s_key[i] = ~KT(0);
        __syncthreads();
        bitonic64(reinterpret_cast<unsigned long long *>(s_key), npow2);
    }
    __syncthreads();
    constexpr KT LOCAL_MASK = K32 ? KT(0x7FF) : KT(0xFFFFFFFFu);
    // each entry's (local pixel, weight) in sorted order: independent loads
#pragma unroll 4
    for (int i = threadIdx.x; i < n; i += T) {
        const uint32_t loc = uint32_t(s_key[i] & LOCAL_MASK);
        const int pix = int(loc) / K, j = int(loc) - pix * K;
        const int64_t pp = int64_t(ty * tile_h + pix / tile_w) * W + tx * tile_w + pix % tile_w;
        s_ent[i] = make_uint2(uint32_t(pix), __float_as_uint(wts[pp * K + j]));
    }
    if (threadIdx.x == 0) s_nseg = 0;
    // segment starts
    uint32_t carry = 0;
    for (int base_i = 0; base_i < n; base_i += T) {
        const int i = base_i + threadIdx.x;
        const uint32_t h = (i < n && (i == 0 || (s_key[i] >> SHIFT) != (s_key[i - 1] >> SHIFT))) ? 1u : 0u;
        uint32_t chunk;
        const uint32_t hi = block_inclusive_scan(h, s_w, chunk);
        if (h) seg[carry + hi - 1] = uint32_t(i);
        carry += chunk;
    }
    if (threadIdx.x == 0) s_nseg = carry;
    __syncthreads();
    const int nseg = int(s_nseg);
    // segment u's partial row goes to slot r.x + u (u < nseg <= r.y - r.x); the
    // slot is recorded in the Gaussian's slot map at this tile's position in
    // its footprint rectangle (row-major, so the map lists its slots in tile order)
    for (int u = threadIdx.x; u < nseg; u += T) {
        const uint32_t gid = uint32_t(s_key[seg[u]] >> SHIFT);
        const uint2 rc = rect[gid];
        const int tx0 = int(rc.x & 0xFFFFu), ty0 = int(rc.x >> 16);
        const int tw = int(rc.y & 0xFFFFu) - tx0 + 1;
        const int64_t i = int64_t(ty - ty0) * tw + (tx - tx0);
        const int64_t at = int64_t(goff[gid]) + i;
        if (tx >= tx0 && ty >= ty0 && i < int64_t(tcount[gid]) && at < X) slotmap[at] = r.x + uint32_t(u);
        // the first tile to select the Gaussian lists it (the order of the
        // lists does not matter: each entry is summed on its own)
        if (atomicExch(&gflag[gid], 1u) == 0u) {
            const bool big = tcount[gid] > uint32_t(kRowsSmall);
            uint32_t *list = lists + (big ? N : 0);
            list[atomicAdd(lists + 2 * N + (big ? 1 : 0), 1u)] = gid;
        }
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    // per-entry (dalpha, dA) sums: lanes take entries b + lane, b + lane + 32, ...
    for (int u = warp; u < nseg; u += T / 32) {
        const int b = int(seg[u]), e = (u + 1 < nseg) ? int(seg[u + 1]) : n;
        float4 sacc = make_float4(0.f, 0.f, 0.f, 0.f);
        for (int i = b + lane; i < e; i += 32) {
            const uint32_t loc = uint32_t(s_key[i] & LOCAL_MASK);
            const int pix = int(loc) / K, j = int(loc) - pix * K;
            const int64_t pp = int64_t(ty * tile_h + pix / tile_w) * W + tx * tile_w + pix % tile_w;
            const float4 ee = E4[pp * K + j];
            sacc.x += ee.x; sacc.y += ee.y; sacc.z += ee.z; sacc.w += ee.w;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            sacc.x += __shfl_xor_sync(0xffffffffu, sacc.x, o);
            sacc.y += __shfl_xor_sync(0xffffffffu, sacc.y, o);
            sacc.z += __shfl_xor_sync(0xffffffffu, sacc.z, o);
            sacc.w += __shfl_xor_sync(0xffffffffu, sacc.w, o);
        }
        if (lane == 0) partial_s[int64_t(r.x) + u] = sacc;
    }
    // the w * g sums, CH (32 or 64) channels at a time
    const int grp = lane >> 3, gl = lane & 7;   // 8-lane group, lane in the group
    constexpr int NWARP = T / 32;
    const int r0 = int(int64_t(n) * warp / NWARP), r1 = int(int64_t(n) * (warp + 1) / NWARP);
    int u_lo = 0;   // the segment holding entry r0: the last u with seg[u] <= r0
    for (int hi = nseg; hi - u_lo > 1;) {
        const int mid = (u_lo + hi) >> 1;
        if (int(seg[mid]) <= r0) u_lo = mid; else hi = mid;
    }
    int c_fail = -1;
    for (int c = 0; c < nchunks; ++c) {
        const int c0 = c * CH;
        const float *gbuf = s_g;
        if (use_tma) {
            if (threadIdx.x == 0) s_ok = tma_mbar_wait(&s_bar[0], uint32_t(c) & 1u, kTmaSpin) ? 1 : 0;
            __syncthreads();
            if (!s_ok) { c_fail = c; break; }
        } else {
            __syncthreads();   // the previous chunk is consumed
            for (int i = threadIdx.x; i < T * (CH / 4); i += T) {
                const int pix = i / (CH / 4), c4 = i - pix * (CH / 4);
                const int gx = tx * tile_w + pix % tile_w, gy = ty * tile_h + pix / tile_w;
                float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
                if (gx < W && gy < H && c0 + c4 * 4 < C)
                    v = *reinterpret_cast<const float4 *>(grad_out + (int64_t(gy) * W + gx) * int64_t(C) + c0 + c4 * 4);
                reinterpret_cast<float4 *>(s_g + pix * CH)[c4] = v;
            }
            __syncthreads();
        }
        // balanced walk: warp w sums entries [w n / 8, (w + 1) n / 8); a segment
        // that crosses a warp boundary is split into pieces, the piece holding
        // its start is completed below with the next warps' pieces, in order.
        // The warp's four 8-lane groups take every fourth entry of a piece
        // (group q: entries b + q, b + q + 4, ...); lane j of a group holds
        // channels 4j .. 4j + 3 (a) and, for 64-channel chunks, 32 + 4j ..
        // 32 + 4j + 3 (b) of the chunk.  The group sums are added as
        // (q0 + q1) + (q2 + q3) at the end of the piece.
        auto walk = [&](int b, int e, float4 &a, float4 &bb) {
            a = make_float4(0.f, 0.f, 0.f, 0.f);
            bb = make_float4(0.f, 0.f, 0.f, 0.f);
            int i = b + grp;
            for (; i + 4 < e; i += 8) {
                const uint2 e0 = s_ent[i], e1 = s_ent[i + 4];
                const float4 *g0 = reinterpret_cast<const float4 *>(gbuf + e0.x * CH);
                const float4 *g1 = reinterpret_cast<const float4 *>(gbuf + e1.x * CH);
                const float4 x0 = g0[gl], x1 = g1[gl];
                const float w0 = __uint_as_float(e0.y), w1 = __uint_as_float(e1.y);
                fma4v(a, w0, x0);
                fma4v(a, w1, x1);
                if (CH == 64) {
                    const float4 y0 = g0[8 + gl], y1 = g1[8 + gl];
                    fma4v(bb, w0, y0);
                    fma4v(bb, w1, y1);
                }
            }
            if (i < e) {
                const uint2 e0 = s_ent[i];
                const float4 *g0 = reinterpret_cast<const float4 *>(gbuf + e0.x * CH);
                const float w0 = __uint_as_float(e0.y);
                fma4v(a, w0, g0[gl]);
                if (CH == 64) fma4v(bb, w0, g0[8 + gl]);
            }
#pragma unroll
            for (int o = 8; o <= 16; o <<= 1) {
                a.x += __shfl_xor_sync(0xffffffffu, a.x, o); a.y += __shfl_xor_sync(0xffffffffu, a.y, o);
                a.z += __shfl_xor_sync(0xffffffffu, a.z, o); a.w += __shfl_xor_sync(0xffffffffu, a.w, o);
                if (CH == 64) {
                    bb.x += __shfl_xor_sync(0xffffffffu, bb.x, o); bb.y += __shfl_xor_sync(0xffffffffu, bb.y, o);
                    bb.z += __shfl_xor_sync(0xffffffffu, bb.z, o); bb.w += __shfl_xor_sync(0xffffffffu, bb.w, o);
                }
            }
        };
        // group 0 stores the piece's 32 or 64 channels
        auto store = [&](int u, const float4 &a, const float4 &bb) {
            if (grp != 0) return;
            float *dst = partial + (int64_t(r.x) + u) * C + c0;
            if (c0 + 4 * gl < C) *reinterpret_cast<float4 *>(dst + 4 * gl) = a;
            if (CH == 64 && c0 + 32 + 4 * gl < C) *reinterpret_cast<float4 *>(dst + 32 + 4 * gl) = bb;
        };
        float4 *pc = s_piece[c & 1];   // [warp][first, last][16 float4]
        int *sf = s_first[c & 1], *sla = s_last[c & 1];
        int first_u = -1, last_u = -1;
        if (r0 < r1) {
            for (int u = u_lo; u < nseg && int(seg[u]) < r1; ++u) {
                const int sb = int(seg[u]), se = (u + 1 < nseg) ? int(seg[u + 1]) : n;
                float4 a, bb;
                walk(max(sb, r0), min(se, r1), a, bb);
                if (sb < r0 || se > r1) {
                    // continues a segment begun by an earlier warp (slot 0), or
                    // begins one that later warps continue (slot 1)
                    const int sl = sb < r0 ? 0 : 1;
                    if (grp == 0) {
                        pc[(warp * 2 + sl) * 16 + gl] = a;
                        pc[(warp * 2 + sl) * 16 + 8 + gl] = bb;
                    }
                    if (sl == 0) first_u = u; else last_u = u;
                } else {
                    store(u, a, bb);
                }
            }
        }
        if (lane == 0) {
            sf[warp] = first_u;
            sla[warp] = last_u;
        }
        __syncthreads();   // the chunk's g is consumed and the pieces are visible
        if (use_tma && threadIdx.x == 0 && c + 1 < nchunks) {
            // refill the buffer while the pieces are combined (the pieces use
            // the other half of the piece buffer in the next chunk)
            tma_expect_tx(&s_bar[0], chunk_bytes);
            tma_load_3d(s_g, &gmap, (c + 1) * CH, tx * tile_w, ty * tile_h, &s_bar[0]);
        }
        if (sla[warp] >= 0) {
            const int u = sla[warp];
            float4 a = pc[(warp * 2 + 1) * 16 + gl], bb = pc[(warp * 2 + 1) * 16 + 8 + gl];
            for (int w2 = warp + 1; w2 < NWARP; ++w2) {
                const int a2 = int(int64_t(n) * w2 / NWARP), b2 = int(int64_t(n) * (w2 + 1) / NWARP);
                if (a2 >= b2) continue;        // an empty range holds no piece
                if (sf[w2] != u) break;
                const float4 v = pc[(w2 * 2) * 16 + gl], vb = pc[(w2 * 2) * 16 + 8 + gl];
                a.x += v.x; a.y += v.y; a.z += v.z; a.w += v.w;
                bb.x += vb.x; bb.y += vb.y; bb.z += vb.z; bb.w += vb.w;
            }
            store(u, a, bb);
        }
    }
    if (c_fail >= 0 && threadIdx.x == 0) {
        // a staging copy did not arrive: report it, and let the copies still in
        // flight (chunk c_fail) land before the CTA exits
        atomicExch(&counters[CNT_STATUS], uint32_t(QR_ERR_DEVICE_TIMEOUT));
        tma_mbar_wait(&s_bar[0], uint32_t(c_fail) & 1u, kTmaSpin);
    }
}

// ------------------------------------------------------------------ 3. per Gaussian
// Each Gaussian's first intersection index (the exclusive prefix of the tile
// counts over Gaussians), from the projection's tile counts and the per-256
// block bases the binning left in the frame -- the arithmetic of the binning's
// own offsets, for every Gaussian.
__global__ void __launch_bounds__(kProjectThreads)
isect_offsets(const uint32_t *__restrict__ tcount, const uint32_t *__restrict__ tsum_base,
              int64_t n, uint32_t *__restrict__ goff, uint32_t *__restrict__ d_nlist) {
    __shared__ uint32_t s_w[32];
    if (blockIdx.x == 0 && threadIdx.x < 2) d_nlist[threadIdx.x] = 0;   // the selected lists start empty
    const int64_t g = int64_t(blockIdx.x) * kProjectThreads + threadIdx.x;
    const uint32_t c = g < n ? tcount[g] : 0u;
    uint32_t tot;
    const uint32_t cinc = block_inclusive_scan(c, s_w, tot);
    if (g < n) goff[g] = tsum_base[blockIdx.x] + cinc - c;
}

// A selected Gaussian's slot map -- one entry per tile of its footprint
// rectangle (row-major, so in tile order), from its first intersection index
// -- holds the slot of its partial row in every tile that selected it and
// 0xFFFFFFFF elsewhere; the tile kernel lists the selected Gaussians, those
// with more than kRowsSmall tiles apart.
// One CTA of NT threads per listed Gaussian: it walks the map NT tiles at a
// time, compacts the found slots in tile order into shared memory, and its
// NW = NT / 32 warps add the rows: warp w takes the 128-channel block w % nb
// (nb = C / 128 rounded up) and, when nb < NW, the rows i = w / nb (mod R),
// R = NW / nb, in order, eight rows in flight; the R partial sums are added in
// subset order at the end.  Warp 0 adds the (dalpha, dA) terms of the found
// slots in tile order.  Channel blocks beyond NW are taken in further rounds.
template <int NT>
__global__ void __launch_bounds__(NT)
bwd_rows(const uint32_t *__restrict__ list, const uint32_t *__restrict__ d_nlist,
         const uint32_t *__restrict__ goff, const uint32_t *__restrict__ tcount,
         const uint32_t *__restrict__ slotmap, int64_t X, const float *__restrict__ partial,
         const float4 *__restrict__ partial_s, int C, float *__restrict__ grad_feat,
         float *__restrict__ grad_alpha, float *__restrict__ grad_conic) {
    constexpr unsigned FULL = 0xffffffffu;
    constexpr int NW = NT / 32;
    __shared__ uint32_t s_slot[NT];
    __shared__ uint32_t s_w[32];
    __shared__ float4 s_acc[NW][32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nb = (C + 127) / 128;
    const int R = nb < NW ? NW / nb : 1;          // row subsets per channel block
    const uint32_t nlist = *d_nlist;
    for (uint32_t wi = blockIdx.x; wi < nlist; wi += gridDim.x) {
        const uint32_t g = list[wi];
        const int64_t m0 = goff[g];
        int64_t nt = tcount[g];
        if (m0 + nt > X) nt = X > m0 ? X - m0 : 0;
        float4 sacc = make_float4(0.f, 0.f, 0.f, 0.f);
        for (int cg = 0; cg < nb; cg += NW) {            // rounds of channel blocks
            const int blk = cg + (R > 1 ? warp % nb : warp);
            const int sub = R > 1 ? warp / nb : 0;
            const bool on = blk < nb && sub < R;
            const int c0 = blk * 128 + lane * 4;
            const bool act = on && c0 < C;
            float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
            for (int64_t base = 0; base < nt; base += NT) {
                const uint32_t slot = base + threadIdx.x < nt ? slotmap[m0 + base + threadIdx.x] : 0xFFFFFFFFu;
                const uint32_t f = slot != 0xFFFFFFFFu ? 1u : 0u;
                uint32_t nf;
                const uint32_t pos = block_inclusive_scan(f, s_w, nf);
                if (f) s_slot[pos - 1] = slot;
                __syncthreads();
                if (cg == 0 && warp == 0) {
                    for (uint32_t i0 = 0; i0 < nf; i0 += 32) {
                        const float4 mine = i0 + lane < nf ? partial_s[s_slot[i0 + lane]] : make_float4(0.f, 0.f, 0.f, 0.f);
                        const int cnt = int(min(32u, nf - i0));
                        for (int q = 0; q < cnt; ++q) {
                            sacc.x += __shfl_sync(FULL, mine.x, q);
                            sacc.y += __shfl_sync(FULL, mine.y, q);
                            sacc.z += __shfl_sync(FULL, mine.z, q);
                            sacc.w += __shfl_sync(FULL, mine.w, q);
                        }
                    }
                }
                if (act) {
                    // this subset's rows: sub, sub + R, sub + 2R, ... of the found list
                    for (uint32_t i = uint32_t(sub); i < nf; i += 8u * uint32_t(R)) {
                        float4 v[8];
#pragma unroll
                        for (int x = 0; x < 8; ++x) {
                            const uint32_t ii = i + uint32_t(x * R);
                            if (ii < nf) v[x] = *reinterpret_cast<const float4 *>(partial + int64_t(s_slot[ii]) * C + c0);
                        }
#pragma unroll
                        for (int x = 0; x < 8; ++x)
                            if (i + uint32_t(x * R) < nf) { acc.x += v[x].x; acc.y += v[x].y; acc.z += v[x].z; acc.w += v[x].w; }
                    }
                }
                __syncthreads();   // s_slot is rewritten by the next step
            }
            // the R subsets of each channel block, added in subset order
            s_acc[warp][lane] = acc;
            __syncthreads();
            if (on && sub == 0 && c0 < C) {
                float4 t = acc;
                for (int q = 1; q < R; ++q) {
                    const float4 o = s_acc[warp + q * nb][lane];
                    t.x += o.x; t.y += o.y; t.z += o.z; t.w += o.w;
                }
                *reinterpret_cast<float4 *>(grad_feat + int64_t(g) * C + c0) = t;
            }
            __syncthreads();
        }
        if (threadIdx.x == 0) {
            if (grad_alpha) grad_alpha[g] = sacc.x;
            if (grad_conic) {
                grad_conic[3 * int64_t(g)] = sacc.y;
                grad_conic[3 * int64_t(g) + 1] = sacc.z;
                grad_conic[3 * int64_t(g) + 2] = sacc.w;
            }
        }
    }
}

int sms_now() {
    int dev = 0, sms = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sms;
}

inline size_t up256(size_t x) { return (x + 255) / 256 * 256; }

// A non-blocking stream per device on which the backward clears its outputs
// while the tile kernel runs (forked from and joined back to the caller's
// stream with events, so the pattern is also valid under graph capture).
cudaStream_t side_stream() {
    constexpr int kMaxDev = 64;
    static cudaStream_t streams[kMaxDev];
    static std::once_flag once[kMaxDev];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDev) return nullptr;
    std::call_once(once[dev], [dev] {
        if (cudaStreamCreateWithFlags(&streams[dev], cudaStreamNonBlocking) != cudaSuccess)
            streams[dev] = nullptr;
    });
    return streams[dev];
}

struct BwdLayout {
    size_t e, partial, partial_s, goff, slotmap, gflag, lists, total;
};

BwdLayout bwd_layout(const qr_frame &f, int C) {
    const size_t P = size_t(num_pixels(f)), K = size_t(f.params.K), X = size_t(f.max_isect);
    BwdLayout L;
    size_t o = 0;
    L.e = o; o = up256(o + P * K * 16);
    L.partial = o; o = up256(o + X * size_t(C) * 4);
    L.partial_s = o; o = up256(o + X * 16);
    L.goff = o; o = up256(o + size_t(f.n) * 4);   // first intersection index per Gaussian
    L.slotmap = o; o = up256(o + X * 4);          // per intersection: partial slot or none
    L.gflag = o; o = up256(o + size_t(f.n) * 4);       // Gaussian listed yet
    L.lists = o; o = up256(o + size_t(f.n) * 8 + 8);   // selected: small list, big list, counts
    L.total = o;
    return L;
}

// vectors of 16 bytes per lane when every lane holds the same number (0: not)
int bwd_vpl(qr_dtype dt, int C) {
    const int cpv = dt == QR_F32 ? 4 : dt == QR_BF16 ? 8 : 16;
    const int nvec = C % cpv == 0 ? C / cpv : 0;
    const int vpl = nvec % 32 == 0 ? nvec / 32 : 0;
    return vpl == 1 || vpl == 2 || vpl == 4 ? vpl : 0;
}

// loss != nullptr: the fused cosine-loss pass (bwd_vpl(dt, C) > 0), g is its output
template <int DT>
void launch_bwd_pixel(const qr_frame &f, const void *feat, const float *scale, int C,
                      const int32_t *ids, const float *w, const uint8_t *cnt, float *g,
                      float4 *E, const CosLossArgs *loss, cudaStream_t s) {
    const int64_t P = num_pixels(f);
    const int64_t warps = P;
    int64_t blocks = (warps * 32 + T - 1) / T;
    const int64_t cap = int64_t(sms_now()) * 8;
    if (blocks > cap) blocks = cap;
    const int vpl = bwd_vpl(qr_dtype(DT), C);
    PixLoss pl{};
    if (loss) pl = PixLoss{loss->F, loss->tgt, loss->mask, loss->term, loss->out2};
    auto go = [&](auto kern) {
        kern<<<unsigned(blocks), T, 0, s>>>(
            slot<float4>(f, S_REC_M), slot<float4>(f, S_REC_C), slot<float>(f, S_REC_A),
            static_cast<const unsigned char *>(feat), scale, C, ids, w, cnt, g, P, f.params.K,
            f.camera.width, f.params.alpha_max, E, pl);
    };
    if (loss) {
        switch (vpl) {
            case 1: go(bwd_pixel<DT, 1, true>); break;
            case 2: go(bwd_pixel<DT, 2, true>); break;
            default: go(bwd_pixel<DT, 4, true>); break;
        }
        return;
    }
    switch (vpl) {
        case 1: go(bwd_pixel<DT, 1, false>); break;
        case 2: go(bwd_pixel<DT, 2, false>); break;
        case 4: go(bwd_pixel<DT, 4, false>); break;
        default: go(bwd_pixel<DT, 0, false>); break;
    }
}

}  // namespace

namespace {

cudaError_t backward_impl(const qr_frame &f, const void *feat, const float *scale, qr_dtype dt,
                          int C, const int32_t *ids, const float *w, const uint8_t *cnt,
                          const float *grad_out, const CosLossArgs *loss, float *grad_feat,
                          float *grad_alpha, float *grad_conic, void *ws, cudaStream_t s) {
    const BwdLayout L = bwd_layout(f, C);
    char *b = static_cast<char *>(ws);
    float4 *E = reinterpret_cast<float4 *>(b + L.e);
    float *partial = reinterpret_cast<float *>(b + L.partial);
    float4 *partial_s = reinterpret_cast<float4 *>(b + L.partial_s);
    uint32_t *goff = reinterpret_cast<uint32_t *>(b + L.goff);
    uint32_t *slotmap = reinterpret_cast<uint32_t *>(b + L.slotmap);
    uint32_t *gflag = reinterpret_cast<uint32_t *>(b + L.gflag);
    uint32_t *lists = reinterpret_cast<uint32_t *>(b + L.lists);
    uint32_t *counters = slot<uint32_t>(f, S_COUNTERS);
    const int tiles = num_tiles(f);
    const int K = f.params.K;
    cudaError_t e = cudaMemsetAsync(slotmap, 0xFF, size_t(f.max_isect) * 4, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(gflag, 0, size_t(f.n) * 4, s);
    if (e != cudaSuccess) return e;
    isect_offsets<<<unsigned((f.n + kProjectThreads - 1) / kProjectThreads), kProjectThreads, 0, s>>>(
        slot<uint32_t>(f, S_TCOUNT), slot<uint32_t>(f, S_BSUM), f.n, goff, lists + 2 * f.n);
    float *g = const_cast<float *>(grad_out);   // written only by the fused loss pass
    switch (dt) {
        case QR_F32: launch_bwd_pixel<QR_F32>(f, feat, scale, C, ids, w, cnt, g, E, loss, s); break;
        case QR_BF16: launch_bwd_pixel<QR_BF16>(f, feat, scale, C, ids, w, cnt, g, E, loss, s); break;
        case QR_FP8E4M3: launch_bwd_pixel<QR_FP8E4M3>(f, feat, scale, C, ids, w, cnt, g, E, loss, s); break;
    }
    if (loss) {
        e = cudaGetLastError();
        if (e == cudaSuccess) e = launch_cos_final(loss->term, num_pixels(f), loss->out2, s);
        if (e != cudaSuccess) return e;
    }
    // rows of Gaussians that no tile selects are zero: clear the outputs on the
    // side stream, overlapping the tile kernel (which is not bandwidth-bound),
    // and join before the rows are written; without a side stream, in order
    cudaStream_t side = side_stream();
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    if (side && (cudaEventCreateWithFlags(&ev_fork, cudaEventDisableTiming) != cudaSuccess ||
                 cudaEventCreateWithFlags(&ev_join, cudaEventDisableTiming) != cudaSuccess)) {
        if (ev_fork) cudaEventDestroy(ev_fork);
        ev_fork = nullptr;
        side = nullptr;
    }
    cudaStream_t zs = s;
    if (side) {
        e = cudaEventRecord(ev_fork, s);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(side, ev_fork, 0);
        if (e != cudaSuccess) {
            cudaEventDestroy(ev_fork);
            cudaEventDestroy(ev_join);
            return e;
        }
        zs = side;
    }
    e = cudaMemsetAsync(grad_feat, 0, size_t(f.n) * size_t(C) * 4, zs);
    if (e == cudaSuccess && grad_alpha) e = cudaMemsetAsync(grad_alpha, 0, size_t(f.n) * 4, zs);
    if (e == cudaSuccess && grad_conic) e = cudaMemsetAsync(grad_conic, 0, size_t(f.n) * 12, zs);
    // the side stream joins the caller's stream again (also on an error path)
    auto join = [&](cudaError_t err) {
        if (!side) return err;
        cudaError_t ej = cudaEventRecord(ev_join, side);
        if (ej == cudaSuccess) ej = cudaStreamWaitEvent(s, ev_join, 0);
        cudaEventDestroy(ev_fork);
        cudaEventDestroy(ev_join);
        side = nullptr;
        return err != cudaSuccess ? err : ej;
    };
    if (e != cudaSuccess) return join(e);
    // per-tile partials; for K <= 8 the tile's rows of g are staged by TMA
    // (3-D boxes {64 channels, tile_w pixels, tile_h rows} of the [H][W][C]
    // gradient) when the driver provides a tensor-map encoder
    int npow2 = 1;
    while (npow2 < 256 * K) npow2 <<= 1;
    const int CH = K <= 8 ? 64 : 32;
    CUtensorMap gmap;
    std::memset(&gmap, 0, sizeof(gmap));
    int use_tma = 0;
    if (K <= 8) {
        EncodeTiled enc = tensor_map_encoder();
        const cuuint64_t dims[3] = {cuuint64_t(C), cuuint64_t(f.camera.width), cuuint64_t(f.camera.height)};
        const cuuint64_t strides[2] = {cuuint64_t(C) * 4, cuuint64_t(C) * 4 * cuuint64_t(f.camera.width)};
        const cuuint32_t box[3] = {cuuint32_t(CH), cuuint32_t(f.params.tile_w), cuuint32_t(f.params.tile_h)};
        const cuuint32_t estr[3] = {1, 1, 1};
        if (enc && enc(&gmap, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float *>(grad_out), dims,
                       strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                       CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS)
            use_tma = 1;
    }
    // One CTA per tile.  With TMA staging the CTA holds one g chunk (64
    // channels x 256 pixels, 64 KB) and reads the E terms from global memory,
    // so two CTAs share an SM and one's sort, gathers and staging waits
    // overlap the other's walk.
    const bool k32 = K <= 8 && f.n < (int64_t(1) << 21);
    const size_t key_bytes = k32 ? 4 : 8;
    const size_t g_off = (size_t(npow2) * key_bytes + size_t(256 * K) * 12 + 1023) & ~size_t(1023);
    const size_t smem = 1024 + g_off + size_t(256) * CH * 4;
    auto tp = [&](auto kern) {
        cudaError_t ee = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
        if (ee != cudaSuccess) return ee;
        ee = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
        if (ee != cudaSuccess) return ee;
        kern<<<unsigned(tiles), T, smem, s>>>(slot<uint2>(f, S_RANGES), f.camera.width,
                                               f.camera.height, f.params.tile_w, f.tiles_x, ids, w,
                                               cnt, E, grad_out, C, K, CH, partial, partial_s,
                                               slot<uint2>(f, S_RECT), slot<uint32_t>(f, S_TCOUNT),
                                               goff, slotmap, f.max_isect, gflag, lists, f.n,
                                               gmap, use_tma, counters);
        return cudaSuccess;
    };
    if (k32) {
        e = K == 1 ? tp(bwd_tile_partials<1, uint32_t>) : K == 2 ? tp(bwd_tile_partials<2, uint32_t>)
          : K <= 4 ? tp(bwd_tile_partials<4, uint32_t>) : K <= 8 ? tp(bwd_tile_partials<8, uint32_t>)
                   : tp(bwd_tile_partials<0, unsigned long long>);
    } else {
        e = K == 1 ? tp(bwd_tile_partials<1, unsigned long long>) : K == 2 ? tp(bwd_tile_partials<2, unsigned long long>)
          : K <= 4 ? tp(bwd_tile_partials<4, unsigned long long>) : K <= 8 ? tp(bwd_tile_partials<8, unsigned long long>)
                   : tp(bwd_tile_partials<0, unsigned long long>);
    }
    e = join(e);
    if (e != cudaSuccess) return e;
    // the selected Gaussians' rows in tile order, over the cleared outputs
    const uint32_t *tcount = slot<uint32_t>(f, S_TCOUNT);
    bwd_rows<256><<<unsigned(sms_now() * 8), 256, 0, s>>>(
        lists, lists + 2 * f.n, goff, tcount, slotmap, f.max_isect, partial, partial_s, C,
        grad_feat, grad_alpha, grad_conic);
    bwd_rows<1024><<<unsigned(sms_now() * 2), 1024, 0, s>>>(
        lists + f.n, lists + 2 * f.n + 1, goff, tcount, slotmap, f.max_isect, partial, partial_s,
        C, grad_feat, grad_alpha, grad_conic);
    count_launch(5);
    return cudaGetLastError();
}

}  // namespace

size_t backward_workspace_bytes(const qr_frame &f, int C) { return bwd_layout(f, C).total; }

size_t backward_cos_workspace_bytes(const qr_frame &f, int C) {
    return bwd_layout(f, C).total + ((size_t(num_pixels(f)) * 4 + 255) & ~size_t(255));
}

cudaError_t launch_backward(const qr_frame &f, const void *feat, const float *scale, qr_dtype dt,
                            int C, const int32_t *ids, const float *w, const uint8_t *cnt,
                            const float *grad_out, float *grad_feat, float *grad_alpha,
                            float *grad_conic, void *ws, cudaStream_t s) {
    return backward_impl(f, feat, scale, dt, C, ids, w, cnt, grad_out, nullptr, grad_feat,
                         grad_alpha, grad_conic, ws, s);
}

cudaError_t launch_backward_cos(const qr_frame &f, const void *feat, const float *scale,
                                qr_dtype dt, int C, const int32_t *ids, const float *w,
                                const uint8_t *cnt, const CosLossArgs &loss, float *grad_feat,
                                float *grad_alpha, float *grad_conic, void *ws, cudaStream_t s) {
    const int64_t P = num_pixels(f);
    if (bwd_vpl(dt, C) == 0) {
        // rows that do not split evenly over the lanes: the loss's own pass first
        cudaError_t e = launch_cosine_loss(loss.F, loss.tgt, loss.mask, P, C, loss.term, loss.out2,
                                           loss.grad_map, s);
        if (e != cudaSuccess) return e;
        return launch_backward(f, feat, scale, dt, C, ids, w, cnt, loss.grad_map, grad_feat,
                               grad_alpha, grad_conic, ws, s);
    }
    cudaError_t e = launch_cos_count(loss.mask, P, loss.out2, s);
    if (e != cudaSuccess) return e;
    return backward_impl(f, feat, scale, dt, C, ids, w, cnt, loss.grad_map, &loss, grad_feat,
                         grad_alpha, grad_conic, ws, s);
}

}  // namespace qr
