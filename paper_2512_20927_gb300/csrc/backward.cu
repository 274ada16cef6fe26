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
//      writes per-entry (dalpha, dA00, dA01, dA11);
//   2. bwd_tile_partials: one CTA per (screen tile, 128-channel slice) sorts
//      the tile's (Gaussian, entry) keys in shared memory and lets each warp
//      reduce one distinct Gaussian's w * g rows in entry order into a partial
//      row, stored at a fixed slot of that tile's intersection range;
//   3. a stable radix sort of the slot keys by Gaussian id;
//   4. bwd_reduce: one warp per Gaussian sums its partials in tile order and
//      writes its gradient row (zeros for unselected Gaussians).
#include <cuda_bf16.h>
#include <cuda_fp8.h>

#include "qr_internal.cuh"

namespace qr {
namespace {

constexpr int T = 256;
constexpr int CHUNK = 128;     // channels per partial-reduction CTA

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
template <int DT>
__global__ void __launch_bounds__(T)
bwd_pixel(const float4 *__restrict__ rec_m, const float4 *__restrict__ rec_w,
          const float *__restrict__ rec_a, const unsigned char *__restrict__ feat,
          const float *__restrict__ fscale, int C, const int32_t *__restrict__ ids,
          const float *__restrict__ wts, const uint8_t *__restrict__ cnt,
          const float *__restrict__ grad_out, int64_t P, int K, int W, float alpha_max,
          float4 *__restrict__ E) {
    constexpr int CPV = VecB<DT>::C, ESZ = VecB<DT>::E;
    constexpr unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const int64_t warp0 = (int64_t(blockIdx.x) * T + threadIdx.x) >> 5;
    const int64_t nw = (int64_t(gridDim.x) * T) >> 5;
    const int nvec = C / CPV;                      // 16-byte vectors per feature row
    const size_t row_bytes = size_t(C) * ESZ;
    for (int64_t p = warp0; p < P; p += nw) {
        const int m = cnt[p];
        if (m == 0) continue;
        const float ux = float(p % W) + 0.5f, uy = float(p / W) + 0.5f;
        const int id = lane < m ? ids[p * K + lane] : 0;
        const float wj = lane < m ? wts[p * K + lane] : 0.f;
        // s_j = g . f_j for every quantile Gaussian j (lane j keeps s_j)
        const float *g = grad_out + p * int64_t(C);
        float s_mine = 0.f;
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

__global__ void __launch_bounds__(T)
bwd_tile_partials(const uint2 *__restrict__ ranges, int W, int H, int tile_w, int tiles_x,
                  const int32_t *__restrict__ ids, const float *__restrict__ wts,
                  const uint8_t *__restrict__ cnt, const float4 *__restrict__ E,
                  const float *__restrict__ grad_out, int C, int K,
                  float *__restrict__ partial, float4 *__restrict__ partial_s,
                  uint32_t *__restrict__ pkey) {
    extern __shared__ unsigned long long s_key[];          // pow2 >= 256*K keys
    __shared__ uint32_t s_w[32];
    __shared__ uint32_t s_nseg;
    const int tile = blockIdx.x;
    const int c0 = blockIdx.y * CHUNK;
    const int tx = tile % tiles_x, ty = tile / tiles_x;
    const int tile_h = T / tile_w;
    const int px = tx * tile_w + threadIdx.x % tile_w, py = ty * tile_h + threadIdx.x / tile_w;
    const bool inside = px < W && py < H;
    const int64_t p = inside ? int64_t(py) * W + px : 0;
    const uint2 r = ranges[tile];
    const int m = inside ? int(cnt[p]) : 0;
    // gather (gid << 32 | local entry) keys
    uint32_t tot;
    const uint32_t inc = block_inclusive_scan(uint32_t(m), s_w, tot);
    const int n = int(tot);
    int npow2 = 1;
    while (npow2 < n) npow2 <<= 1;
    for (int j = 0; j < m; ++j)
        s_key[inc - m + j] = (static_cast<unsigned long long>(uint32_t(ids[p * K + j])) << 32) |
                             uint32_t(threadIdx.x * K + j);
    for (int i = n + threadIdx.x; i < npow2; i += T) s_key[i] = ~0ull;
    __syncthreads();
    if (n > 1) bitonic64(s_key, npow2);
    // segment heads -> segment starts stored after the keys
    uint32_t *seg = reinterpret_cast<uint32_t *>(s_key + npow2);
    if (threadIdx.x == 0) s_nseg = 0;
    __syncthreads();
    uint32_t carry = 0;
    for (int base = 0; base < n; base += T) {
        const int i = base + threadIdx.x;
        const uint32_t h = (i < n && (i == 0 || (s_key[i] >> 32) != (s_key[i - 1] >> 32))) ? 1u : 0u;
        uint32_t chunk;
        const uint32_t hi = block_inclusive_scan(h, s_w, chunk);
        if (h) seg[carry + hi - 1] = uint32_t(i);
        carry += chunk;
    }
    if (threadIdx.x == 0) s_nseg = carry;
    __syncthreads();
    const int nseg = int(s_nseg);
    if (blockIdx.y == 0) {
        for (int u = threadIdx.x; u < int(r.y - r.x); u += T)
            pkey[r.x + u] = u < nseg ? uint32_t(s_key[seg[u]] >> 32) : 0xFFFFFFFFu;
    }
    // each warp reduces one distinct Gaussian's rows of this channel slice
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int cl = c0 + lane * 4;
    const bool has_c = cl < C;
    const int tile_x0 = tx * tile_w, tile_y0 = ty * tile_h;
    for (int u = warp; u < nseg; u += T / 32) {
        const int b = int(seg[u]), e = (u + 1 < nseg) ? int(seg[u + 1]) : n;
        float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
        float4 sacc = make_float4(0.f, 0.f, 0.f, 0.f);
        for (int i = b; i < e; ++i) {
            const uint32_t loc = uint32_t(s_key[i]);
            const int pix = int(loc) / K, j = int(loc) % K;
            const int64_t pp = int64_t(tile_y0 + pix / tile_w) * W + tile_x0 + pix % tile_w;
            const float w = wts[pp * K + j];
            if (has_c) {
                const float4 gg = *reinterpret_cast<const float4 *>(grad_out + pp * int64_t(C) + cl);
                acc.x = fmaf(w, gg.x, acc.x); acc.y = fmaf(w, gg.y, acc.y);
                acc.z = fmaf(w, gg.z, acc.z); acc.w = fmaf(w, gg.w, acc.w);
            }
            if (blockIdx.y == 0) {
                const float4 ee = E[pp * K + j];
                sacc.x += ee.x; sacc.y += ee.y; sacc.z += ee.z; sacc.w += ee.w;
            }
        }
        const int64_t slot = int64_t(r.x) + u;
        if (has_c) *reinterpret_cast<float4 *>(partial + slot * C + cl) = acc;
        if (blockIdx.y == 0 && lane == 0) partial_s[slot] = sacc;
    }
}

__global__ void __launch_bounds__(T)
iota_kernel(uint32_t *v, const uint32_t *__restrict__ d_n) {
    const uint32_t n = *d_n;
    for (uint32_t i = blockIdx.x * T + threadIdx.x; i < n; i += gridDim.x * T) v[i] = i;
}

// ------------------------------------------------------------------ 3-4. per Gaussian
__global__ void __launch_bounds__(T)
gauss_ranges(const uint32_t *__restrict__ key, const uint32_t *__restrict__ d_n, int64_t N,
             uint2 *__restrict__ gr) {
    const uint32_t n = *d_n;
    for (uint32_t i = blockIdx.x * T + threadIdx.x; i < n; i += gridDim.x * T) {
        const uint32_t k = key[i];
        if (int64_t(k) >= N) continue;
        if (i == 0 || key[i - 1] != k) gr[k].x = i;
        if (i + 1 == n || key[i + 1] != k) gr[k].y = i + 1;
    }
}

__global__ void __launch_bounds__(T)
bwd_reduce(const uint2 *__restrict__ gr, const uint32_t *__restrict__ slot_of,
           const float *__restrict__ partial, const float4 *__restrict__ partial_s, int64_t N,
           int C, float *__restrict__ grad_feat, float *__restrict__ grad_alpha,
           float *__restrict__ grad_conic) {
    const int lane = threadIdx.x & 31;
    const int64_t warp0 = (int64_t(blockIdx.x) * T + threadIdx.x) >> 5;
    const int64_t nw = (int64_t(gridDim.x) * T) >> 5;
    for (int64_t u = warp0; u < N; u += nw) {
        const uint2 r = gr[u];
        float *out = grad_feat + u * int64_t(C);
        for (int c = lane * 4; c < C; c += 128) {
            float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
            for (uint32_t i = r.x; i < r.y; ++i) {
                const float4 v = *reinterpret_cast<const float4 *>(partial + int64_t(slot_of[i]) * C + c);
                acc.x += v.x; acc.y += v.y; acc.z += v.z; acc.w += v.w;
            }
            *reinterpret_cast<float4 *>(out + c) = acc;
        }
        if (lane == 0) {
            float4 s = make_float4(0.f, 0.f, 0.f, 0.f);
            for (uint32_t i = r.x; i < r.y; ++i) {
                const float4 v = partial_s[slot_of[i]];
                s.x += v.x; s.y += v.y; s.z += v.z; s.w += v.w;
            }
            if (grad_alpha) grad_alpha[u] = s.x;
            if (grad_conic) {
                grad_conic[3 * u] = s.y;
                grad_conic[3 * u + 1] = s.z;
                grad_conic[3 * u + 2] = s.w;
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

struct BwdLayout {
    size_t e, partial, partial_s, key0, key1, val0, val1, hist, digitsum, granges, total;
};

BwdLayout bwd_layout(const qr_frame &f, int C) {
    const size_t P = size_t(num_pixels(f)), K = size_t(f.params.K), X = size_t(f.max_isect);
    const size_t N = size_t(f.n);
    BwdLayout L;
    size_t o = 0;
    L.e = o; o = up256(o + P * K * 16);
    L.partial = o; o = up256(o + X * size_t(C) * 4);
    L.partial_s = o; o = up256(o + X * 16);
    L.key0 = o; o = up256(o + X * 4);
    L.key1 = o; o = up256(o + X * 4);
    L.val0 = o; o = up256(o + X * 4);
    L.val1 = o; o = up256(o + X * 4);
    L.hist = o; o = up256(o + size_t(1 << kRadixBitsMax) * kSortMaxBlocks * 4);
    L.digitsum = o; o = up256(o + size_t(1 << kRadixBitsMax) * 4);
    L.granges = o; o = up256(o + N * 8 + 8);
    L.total = o;
    return L;
}

template <int DT>
void launch_bwd_pixel(const qr_frame &f, const void *feat, const float *scale, int C,
                      const int32_t *ids, const float *w, const uint8_t *cnt, const float *g,
                      float4 *E, cudaStream_t s) {
    const int64_t P = num_pixels(f);
    const int64_t warps = P;
    int64_t blocks = (warps * 32 + T - 1) / T;
    const int64_t cap = int64_t(sms_now()) * 8;
    if (blocks > cap) blocks = cap;
    bwd_pixel<DT><<<unsigned(blocks), T, 0, s>>>(
        slot<float4>(f, S_REC_M), slot<float4>(f, S_REC_C), slot<float>(f, S_REC_A),
        static_cast<const unsigned char *>(feat), scale, C, ids, w, cnt, g, P, f.params.K,
        f.camera.width, f.params.alpha_max, E);
}

}  // namespace

size_t backward_workspace_bytes(const qr_frame &f, int C) { return bwd_layout(f, C).total; }

cudaError_t launch_backward(const qr_frame &f, const void *feat, const float *scale, qr_dtype dt,
                            int C, const int32_t *ids, const float *w, const uint8_t *cnt,
                            const float *grad_out, float *grad_feat, float *grad_alpha,
                            float *grad_conic, void *ws, cudaStream_t s) {
    const BwdLayout L = bwd_layout(f, C);
    char *b = static_cast<char *>(ws);
    float4 *E = reinterpret_cast<float4 *>(b + L.e);
    float *partial = reinterpret_cast<float *>(b + L.partial);
    float4 *partial_s = reinterpret_cast<float4 *>(b + L.partial_s);
    uint32_t *key0 = reinterpret_cast<uint32_t *>(b + L.key0);
    uint32_t *key1 = reinterpret_cast<uint32_t *>(b + L.key1);
    uint32_t *val0 = reinterpret_cast<uint32_t *>(b + L.val0);
    uint32_t *val1 = reinterpret_cast<uint32_t *>(b + L.val1);
    uint32_t *hist = reinterpret_cast<uint32_t *>(b + L.hist);
    uint32_t *digitsum = reinterpret_cast<uint32_t *>(b + L.digitsum);
    uint2 *gr = reinterpret_cast<uint2 *>(b + L.granges);
    uint32_t *counters = slot<uint32_t>(f, S_COUNTERS);
    const int tiles = num_tiles(f);
    const int K = f.params.K;
    cudaError_t e = cudaMemsetAsync(gr, 0, size_t(f.n) * 8 + 8, s);
    if (e != cudaSuccess) return e;
    if (grad_alpha) e = cudaMemsetAsync(grad_alpha, 0, size_t(f.n) * 4, s);
    if (e == cudaSuccess && grad_conic) e = cudaMemsetAsync(grad_conic, 0, size_t(f.n) * 12, s);
    if (e != cudaSuccess) return e;
    switch (dt) {
        case QR_F32: launch_bwd_pixel<QR_F32>(f, feat, scale, C, ids, w, cnt, grad_out, E, s); break;
        case QR_BF16: launch_bwd_pixel<QR_BF16>(f, feat, scale, C, ids, w, cnt, grad_out, E, s); break;
        case QR_FP8E4M3: launch_bwd_pixel<QR_FP8E4M3>(f, feat, scale, C, ids, w, cnt, grad_out, E, s); break;
    }
    // per-tile partials
    int npow2 = 1;
    while (npow2 < 256 * K) npow2 <<= 1;
    const size_t smem = size_t(npow2) * 8 + size_t(256 * K) * 4;
    e = cudaFuncSetAttribute(bwd_tile_partials, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    if (e != cudaSuccess) return e;
    dim3 grid(unsigned(tiles), unsigned((C + CHUNK - 1) / CHUNK));
    bwd_tile_partials<<<grid, T, smem, s>>>(slot<uint2>(f, S_RANGES), f.camera.width,
                                            f.camera.height, f.params.tile_w, f.tiles_x, ids, w,
                                            cnt, E, grad_out, C, K, partial, partial_s, key0);
    // stable sort of the slots by Gaussian id (ids < n; unused slots carry 0xFFFFFFFF)
    const uint32_t *d_x = counters + CNT_SORT_N;
    iota_kernel<<<sms_now() * 4, T, 0, s>>>(val0, d_x);
    int in_b = 0;
    e = radix_sort_pairs(key0, val0, key1, val1, d_x, f.max_isect, 0,
                         tile_bits_for(int(f.n + 1 > 2 ? f.n + 1 : 2)), hist, digitsum,
                         f.sort_blocks, &in_b, s);
    if (e != cudaSuccess) return e;
    const uint32_t *skey = in_b ? key1 : key0;
    const uint32_t *sval = in_b ? val1 : val0;
    gauss_ranges<<<sms_now() * 4, T, 0, s>>>(skey, d_x, f.n, gr);
    int64_t blocks = (f.n * 32 + T - 1) / T;
    const int64_t cap = int64_t(sms_now()) * 16;
    if (blocks > cap) blocks = cap;
    if (blocks < 1) blocks = 1;
    bwd_reduce<<<unsigned(blocks), T, 0, s>>>(gr, sval, partial, partial_s, f.n, C, grad_feat,
                                              grad_alpha, grad_conic);
    count_launch(5);
    return cudaGetLastError();
}

}  // namespace qr
