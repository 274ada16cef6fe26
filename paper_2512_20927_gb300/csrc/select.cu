// K5a: the selection half of Algorithm 1 (Sec. 4.2, "sampling quantile
// Gaussians") for every pixel.
//
// Per pixel, front to back over its tile's depth-ordered list:
//   alpha' = min(alpha_max, alpha exp(-q/2)); entries with alpha' < alpha_min
//   are not members of I and leave T unchanged;
//   T_test = T (1 - alpha');
//   if T_test < tau_k (tau_k = (K-k)/(K+1), the boundary 1-(k+1)/(K+1)):
//       keep the Gaussian with weight w = T^Q alpha', T^Q *= 1 - alpha',
//       advance k past every boundary T_test is below;
//   stop once T_test < 1/(K+1); otherwise T = T_test.
// Outputs are the kept ids in depth order and the weights divided by
// 1 - T^Q (the normalisation step folded into the weights).
//
// GB300 design: one CTA per screen tile (256 threads, one per pixel).  The
// tile's list is staged through shared memory 256 entries at a time (gid,
// projected mean hi/lo, conic axes, opacity: 40 B each) with one coalesced load
// per thread; every pixel then reads the staged entries as broadcasts.  The
// walk is scalar FP32 (one exp per pixel-entry pair); a CTA stops loading as
// soon as all of its pixels have stopped (__syncthreads_count).  Kept
// (id, weight) pairs go to per-thread shared-memory slots [K][256] so no
// dynamically indexed register array spills, then are written out once.
#include "qr_internal.cuh"

namespace qr {
namespace {

constexpr int kThreads = 256;

__global__ void __launch_bounds__(kThreads)
select_kernel(const float4 *__restrict__ rec_m, const float4 *__restrict__ rec_w,
              const float *__restrict__ rec_a, const float *__restrict__ rec_h,
              const uint32_t *__restrict__ isect_gid, const uint2 *__restrict__ ranges, int W,
              int H, int tile_w, int tiles_x, int K, float alpha_min, float alpha_max,
              int32_t *__restrict__ ids, float *__restrict__ wout, uint8_t *__restrict__ cnt) {
    __shared__ float4 s_m[kThreads];
    __shared__ float4 s_c[kThreads];
    __shared__ float s_a[kThreads];
    __shared__ float s_h[kThreads];
    __shared__ uint32_t s_g[kThreads];
    extern __shared__ unsigned char s_dyn[];
    int32_t *s_ids = reinterpret_cast<int32_t *>(s_dyn);              // [K][256]
    float *s_w = reinterpret_cast<float *>(s_dyn) + K * kThreads;     // [K][256]

    const int tile = blockIdx.x;
    const int tx = tile % tiles_x, ty = tile / tiles_x;
    const int tile_h = kThreads / tile_w;
    const int lx = threadIdx.x % tile_w, ly = threadIdx.x / tile_w;
    const int px = tx * tile_w + lx, py = ty * tile_h + ly;
    const bool inside = px < W && py < H;
    const float ux = float(px) + 0.5f, uy = float(py) + 0.5f;
    const uint2 range = ranges[tile];

    const float tau_stop = __fdiv_rn(1.0f, float(K + 1));
    float T = 1.0f, TQ = 1.0f;
    int k = 0, m = 0;
    float thr = __fdiv_rn(float(K), float(K + 1));
    bool done = !inside;

    for (uint32_t b = range.x; b < range.y; b += kThreads) {
        if (__syncthreads_count(done) == kThreads) break;
        const uint32_t idx = b + threadIdx.x;
        if (idx < range.y) {
            const uint32_t g = isect_gid[idx];
            s_g[threadIdx.x] = g;
            s_m[threadIdx.x] = rec_m[g];
            s_c[threadIdx.x] = rec_w[g];
            s_a[threadIdx.x] = rec_a[g];
            s_h[threadIdx.x] = rec_h[g];
        }
        __syncthreads();
        const int nb = int(min(uint32_t(kThreads), range.y - b));
        if (!done) {
            for (int j = 0; j < nb; ++j) {
                const float4 mm = s_m[j];
                const float4 cc = s_c[j];
                const PixelTerm pt = eval_half_q(ux, uy, mm, cc);
                if (pt.half_q > s_h[j]) continue;          // alpha' < alpha_min for certain
                const float a = eval_alpha(s_a[j], pt.half_q, alpha_max);
                if (a < alpha_min) continue;
                const float Tt = T * (1.0f - a);
                if (Tt < thr) {
                    s_ids[m * kThreads + threadIdx.x] = int32_t(s_g[j]);
                    s_w[m * kThreads + threadIdx.x] = TQ * a;
                    ++m;
                    TQ = TQ * (1.0f - a);
                    do {
                        ++k;
                        thr = (k < K) ? __fdiv_rn(float(K - k), float(K + 1)) : -1.0f;
                    } while (Tt < thr);
                }
                if (Tt < tau_stop) {
                    done = true;
                    break;
                }
                T = Tt;
            }
        }
    }
    if (!inside) return;
    const int64_t p = int64_t(py) * W + px;
    const float D = 1.0f - TQ;
    for (int j = 0; j < K; ++j) {
        const bool has = j < m;
        ids[p * K + j] = has ? s_ids[j * kThreads + threadIdx.x] : -1;
        wout[p * K + j] = has ? __fdiv_rn(s_w[j * kThreads + threadIdx.x], D) : 0.0f;
    }
    cnt[p] = uint8_t(m);
}

}  // namespace

cudaError_t launch_select(const qr_frame &f, int32_t *ids, float *w, uint8_t *cnt,
                          cudaStream_t s) {
    const int tiles = num_tiles(f);
    if (tiles == 0) return cudaSuccess;
    const int K = f.params.K;
    const size_t dyn = size_t(K) * kThreads * 8;
    if (dyn > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(select_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             int(dyn));
        if (e != cudaSuccess) return e;
    }
    select_kernel<<<tiles, kThreads, dyn, s>>>(
        slot<float4>(f, S_REC_M), slot<float4>(f, S_REC_C), slot<float>(f, S_REC_A), slot<float>(f, S_REC_H),
        slot<uint32_t>(f, S_IGID),
        slot<uint2>(f, S_RANGES), f.camera.width, f.camera.height, f.params.tile_w, f.tiles_x, K,
        f.params.alpha_min, f.params.alpha_max, ids, w, cnt);
    count_launch();
    return cudaGetLastError();
}

}  // namespace qr
