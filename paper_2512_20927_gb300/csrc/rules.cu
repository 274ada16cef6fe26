// The two other select rules of the paper, behind the same outputs as the
// Algorithm 1 selection (ids [P][K] in depth order, normalised weights
// [P][K], counts [P]), so the blend serves all three:
//
//   top-K (Sec. 4.2 and the complexity table, the renderer Q-Render is
//   compared against): the K largest Eq. 1 weights w = T alpha' of the dense
//   walk (same alpha' rules, stop before T would fall below T_min), equal
//   weights keeping the earlier entry, blended with their weights divided by
//   the kept sum;
//
//   Stratified-K (App. E): pass 1 walks the list as Eq. 1 does and takes the
//   mean mu and standard deviation sigma of the transmittances after each
//   blended Gaussian; the K boundaries are spaced uniformly in the
//   probability of N(mu, sigma^2) over the transmittance interval [0, 1]
//   and mapped back (tau_k = mu + sigma Phi^-1(u_lo + (u_hi - u_lo)(1 -
//   k/(K+1))), u_lo = Phi(-mu/sigma), u_hi = Phi((1-mu)/sigma)); pass 2 is
//   Algorithm 1 with tau_k in place of 1 - k/(K+1).
//
// (App. C's Riemann-weight form of Algorithm 1 keeps Algorithm 1's
// selection, so it runs in the selection kernel itself, select.cu.)
//
// GB300 design: one CTA per screen tile, one thread per pixel (256).  The
// tile's depth-ordered list is staged through shared memory 256 records at
// a time; each warp culls 32 staged entries at once against its box of
// pixel centres (the test the Algorithm 1 selection uses), and walks the
// survivors from the ballot mask.  Every pixel evaluates alpha' and the
// transmittance exactly as the dense blend does, so the walks agree with it
// bit for bit.
//   * top-K keeps its candidates in per-pixel shared-memory slots (weight and
//     list position); a strictly larger weight replaces the smallest (latest
//     among equal) one.  Once fl(T alpha_max) is no larger than the smallest
//     kept weight, no later entry can enter (T only falls and alpha' <=
//     alpha_max), so the pixel stops early without changing the result.
//   * Stratified-K sums T and T^2 in compensated double-FP32 arithmetic, forms
//     mu and sigma from them, and the boundaries with the FP32 normal CDF and
//     its inverse (normcdff, normcdfinvf); the boundaries sit in shared memory
//     for pass 2, which re-walks the list.
#include "qr_internal.cuh"

namespace qr {
namespace {

constexpr int kPix = 256;
constexpr int kThreads = 256;
constexpr int kBatch = 256;

enum { kTopK = 1, kStratified = 2 };

struct Stage {
    float4 *m, *c;
    float *a, *h;
};

// Walks the tile's list for this thread's pixel: stages records, culls them
// per warp against the warp's pixel box and calls visit(pos, alpha') for
// every member entry (alpha' >= alpha_min) in list order until the pixel is
// done.  visit returns true when the pixel has finished its walk.  All
// threads of the CTA must call it.
template <typename Visit>
__device__ __forceinline__ void walk_list(const float4 *__restrict__ rec_m,
                                          const float4 *__restrict__ rec_w,
                                          const float *__restrict__ rec_a,
                                          const float *__restrict__ rec_h,
                                          const uint32_t *__restrict__ isect_gid, uint2 range,
                                          const Stage &st, float ux, float uy, float bx0,
                                          float bx1, float by0, float by1, float alpha_min,
                                          float alpha_max, bool &done, Visit visit) {
    constexpr unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    for (uint32_t b = range.x; b < range.y; b += kBatch) {
        if (__syncthreads_count(done) == kThreads) break;
        if (b + threadIdx.x < range.y) {
            const uint32_t g = isect_gid[b + threadIdx.x];
            st.m[threadIdx.x] = rec_m[g];
            st.c[threadIdx.x] = rec_w[g];
            st.a[threadIdx.x] = rec_a[g];
            st.h[threadIdx.x] = rec_h[g];
        }
        __syncthreads();
        const int nb = int(min(uint32_t(kBatch), range.y - b));
        for (int c0 = 0; c0 < nb; c0 += 32) {
            if (__all_sync(FULL, done)) break;
            const int jl = c0 + lane;
            bool pass = false;
            if (jl < nb)
                pass = !(box_min_half_q(st.m[jl], st.c[jl], bx0, bx1, by0, by1) * 0.999f >
                         st.h[jl] + 1e-3f);
            unsigned todo = __ballot_sync(FULL, pass);
            while (todo && !done) {
                const int j = c0 + __ffs(todo) - 1;
                todo &= todo - 1u;
                const PixelTerm pt = eval_half_q(ux, uy, st.m[j], st.c[j]);
                if (pt.half_q > st.h[j]) continue;
                const float a = eval_alpha(st.a[j], pt.half_q, alpha_max);
                if (a < alpha_min) continue;
                done = visit(b + uint32_t(j), a);
            }
        }
        __syncthreads();   // the stage is rewritten by the next batch
    }
}

template <int RULE>
__global__ void __launch_bounds__(kThreads)
rule_kernel(const float4 *__restrict__ rec_m, const float4 *__restrict__ rec_w,
            const float *__restrict__ rec_a, const float *__restrict__ rec_h,
            const uint32_t *__restrict__ isect_gid, const uint2 *__restrict__ ranges, int W,
            int H, int tile_w, int tiles_x, int K, float alpha_min, float alpha_max,
            float T_min, int32_t *__restrict__ ids, float *__restrict__ wout,
            uint8_t *__restrict__ cnt, float *__restrict__ tau_out) {
    pdl_wait();
    __shared__ float4 s_m[kBatch];
    __shared__ float4 s_c[kBatch];
    __shared__ float s_a[kBatch];
    __shared__ float s_h[kBatch];
    extern __shared__ unsigned char s_dyn[];
    const int KS = K | 1;   // odd stride: a thread's slots fall in their own banks
    uint32_t *s_key = reinterpret_cast<uint32_t *>(s_dyn);                 // [256][KS]
    float *s_w = reinterpret_cast<float *>(s_dyn) + KS * kPix;             // [256][KS]
    float *s_tau = reinterpret_cast<float *>(s_dyn) + 2 * KS * kPix;       // [256][KS] (stratified)
    const Stage st{s_m, s_c, s_a, s_h};

    const int tile = blockIdx.x;
    const int tx = tile % tiles_x, ty = tile / tiles_x;
    const int tile_h = kPix / tile_w;
    const int lx = threadIdx.x % tile_w, ly = threadIdx.x / tile_w;
    const int px = tx * tile_w + lx, py = ty * tile_h + ly;
    const bool inside = px < W && py < H;
    const float ux = float(px) + 0.5f, uy = float(py) + 0.5f;
    const uint2 range = ranges[tile];
    uint32_t *my_key = s_key + threadIdx.x * KS;
    float *my_w = s_w + threadIdx.x * KS;
    float *my_tau = s_tau + threadIdx.x * KS;

    constexpr unsigned FULL = 0xffffffffu;
    float bx0 = ux, bx1 = ux, by0 = uy, by1 = uy;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        bx0 = fminf(bx0, __shfl_xor_sync(FULL, bx0, o));
        bx1 = fmaxf(bx1, __shfl_xor_sync(FULL, bx1, o));
        by0 = fminf(by0, __shfl_xor_sync(FULL, by0, o));
        by1 = fmaxf(by1, __shfl_xor_sync(FULL, by1, o));
    }

    int m = 0;          // kept entries
    float D = 0.0f;     // normaliser
    if (RULE == kTopK) {
        // ---- one dense walk keeping the K largest weights
        float T = 1.0f, wmin = 0.0f;
        int smin = 0;
        bool done = !inside;
        walk_list(rec_m, rec_w, rec_a, rec_h, isect_gid, range, st, ux, uy, bx0, bx1, by0, by1,
                  alpha_min, alpha_max, done, [&](uint32_t pos, float a) -> bool {
                      const float Tt = __fmul_rn(T, __fsub_rn(1.0f, a));
                      if (T_min > 0.0f && Tt < T_min) return true;
                      const float w = __fmul_rn(T, a);
                      T = Tt;
                      if (m < K) {
                          my_key[m] = pos;
                          my_w[m] = w;
                          ++m;
                          if (m < K) return false;
                      } else if (w > wmin) {
                          my_key[smin] = pos;
                          my_w[smin] = w;
                      } else {
                          return __fmul_rn(T, alpha_max) <= wmin;
                      }
                      // the smallest kept weight, the latest entry among equal ones
                      smin = 0;
                      for (int j = 1; j < K; ++j)
                          if (my_w[j] < my_w[smin] ||
                              (my_w[j] == my_w[smin] && my_key[j] > my_key[smin]))
                              smin = j;
                      wmin = my_w[smin];
                      return __fmul_rn(T, alpha_max) <= wmin;
                  });
        // depth order (list position), then the kept sum in that order
        for (int i = 1; i < m; ++i) {
            const uint32_t kk = my_key[i];
            const float ww = my_w[i];
            int j = i;
            while (j > 0 && my_key[j - 1] > kk) {
                my_key[j] = my_key[j - 1];
                my_w[j] = my_w[j - 1];
                --j;
            }
            my_key[j] = kk;
            my_w[j] = ww;
        }
        for (int j = 0; j < m; ++j) D = __fadd_rn(D, my_w[j]);
        for (int j = 0; j < m; ++j) my_key[j] = isect_gid[my_key[j]];
    } else {
        // ---- pass 1: transmittance statistics of the dense walk
        float T = 1.0f;
        df s1 = df_from(0.0f), s2 = df_from(0.0f);
        int nb = 0;
        bool done = !inside;
        walk_list(rec_m, rec_w, rec_a, rec_h, isect_gid, range, st, ux, uy, bx0, bx1, by0, by1,
                  alpha_min, alpha_max, done, [&](uint32_t, float a) -> bool {
                      const float Tt = __fmul_rn(T, __fsub_rn(1.0f, a));
                      if (T_min > 0.0f && Tt < T_min) return true;
                      T = Tt;
                      s1 = df_add_f(s1, T);
                      s2 = df_add(s2, df_two_prod(T, T));
                      ++nb;
                      return false;
                  });
        // ---- the boundaries
        if (nb >= 2) {
            const df n = df_from(float(nb));
            const df mu2 = df_div(s1, n);
            const df var = df_sub(df_div(s2, n), df_mul(mu2, mu2));
            const float mu = mu2.hi;
            const float sigma = df_sqrt(var).hi;
            const float zlo = __fdiv_rn(-mu, sigma);
            const float zhi = __fdiv_rn(__fsub_rn(1.0f, mu), sigma);
            const float ulo = normcdff(zlo), uhi = normcdff(zhi);
            const float d = __fsub_rn(uhi, ulo);
            for (int k = 1; k <= K; ++k) {
                const float c = __fdiv_rn(float(K + 1 - k), float(K + 1));
                const float z = normcdfinvf(__fmaf_rn(d, c, ulo));
                my_tau[k - 1] = __fmaf_rn(sigma, z, mu);
            }
        } else {
            for (int k = 1; k <= K; ++k) my_tau[k - 1] = __fdiv_rn(float(K + 1 - k), float(K + 1));
        }
        // ---- pass 2: Algorithm 1 with the boundaries tau_k
        float T2 = 1.0f, TQ = 1.0f;
        int k = 0;
        const float tau_stop = my_tau[K - 1];
        bool done2 = !inside;
        walk_list(rec_m, rec_w, rec_a, rec_h, isect_gid, range, st, ux, uy, bx0, bx1, by0, by1,
                  alpha_min, alpha_max, done2, [&](uint32_t pos, float a) -> bool {
                      const float Tt = __fmul_rn(T2, __fsub_rn(1.0f, a));
                      if (k < K && Tt < my_tau[k]) {
                          my_key[m] = isect_gid[pos];
                          my_w[m] = __fmul_rn(TQ, a);
                          ++m;
                          TQ = __fmul_rn(TQ, __fsub_rn(1.0f, a));
                          do {
                              ++k;
                          } while (k < K && Tt < my_tau[k]);
                      }
                      if (Tt < tau_stop) return true;
                      T2 = Tt;
                      return false;
                  });
        D = __fsub_rn(1.0f, TQ);
    }

    // ---- outputs (a pixel outside the image writes nothing)
    if (inside) {
        const int64_t p = int64_t(py) * W + px;
        for (int j = 0; j < K; ++j) {
            const bool has = j < m;
            ids[p * K + j] = has ? int32_t(my_key[j]) : -1;
            wout[p * K + j] = has ? __fdiv_rn(my_w[j], D) : 0.0f;
        }
        cnt[p] = uint8_t(m);
        if (RULE == kStratified && tau_out)
            for (int j = 0; j < K; ++j) tau_out[p * K + j] = my_tau[j];
    }
}

}  // namespace

cudaError_t launch_select_rule(const qr_frame &f, int rule, int32_t *ids, float *w, uint8_t *cnt,
                               float *tau, cudaStream_t s) {
    const int tiles = num_tiles(f);
    if (tiles == 0) return cudaSuccess;
    const int K = f.params.K;
    const size_t dyn = size_t(K | 1) * kPix * 4 * (rule == kStratified ? 3 : 2);
    auto go = [&](auto kern) -> cudaError_t {
        if (dyn > 48 * 1024) {
            const cudaError_t e =
                cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(dyn));
            if (e != cudaSuccess) return e;
        }
        return pdl_launch(kern, dim3(tiles), dim3(kThreads), dyn, s,
                          (const float4 *)slot<float4>(f, S_REC_M),
                          (const float4 *)slot<float4>(f, S_REC_C),
                          (const float *)slot<float>(f, S_REC_A),
                          (const float *)slot<float>(f, S_REC_H),
                          (const uint32_t *)slot<uint32_t>(f, S_IGID),
                          (const uint2 *)slot<uint2>(f, S_RANGES), f.camera.width,
                          f.camera.height, f.params.tile_w, f.tiles_x, K, f.params.alpha_min,
                          f.params.alpha_max, f.params.T_min, ids, w, cnt, tau);
    };
    const cudaError_t e = rule == kTopK ? go(rule_kernel<kTopK>) : go(rule_kernel<kStratified>);
    count_launch();
    return e != cudaSuccess ? e : cudaGetLastError();
}

}  // namespace qr
