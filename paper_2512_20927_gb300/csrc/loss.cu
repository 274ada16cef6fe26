// Cosine loss of the differentiation workload (not in the paper, whose loss is
// the contrastive Eq. 2 on CLIP targets): L = mean over pixels with at least
// one quantile Gaussian of 1 - cos(F_p, t_p), cos = F.t / (max(|F|,eps) max(|t|,eps)),
// and its gradient dL/dF.  Deterministic: the covered pixels are counted
// first (1/n), one pass writes every pixel's term and its gradient row already
// scaled by 1/n, and one CTA sums the terms in a fixed order.
#include "qr_internal.cuh"

namespace qr {
namespace {

constexpr int T = 256;

// Number of covered pixels of [i0, P) strided by the CTA, eight independent
// loads in flight per thread.
__device__ __forceinline__ unsigned long long count_covered(const uint8_t *__restrict__ counts,
                                                            int64_t P) {
    unsigned long long n = 0;
    const int64_t step = blockDim.x;
    int64_t i = threadIdx.x;
    for (; i + 7 * step < P; i += 8 * step) {
        uint32_t c[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) c[u] = counts[i + u * step];
#pragma unroll
        for (int u = 0; u < 8; ++u) n += c[u] > 0;
    }
    for (; i < P; i += step) n += counts[i] > 0;
    return n;
}

// Number of covered pixels -> 1/n (out[1]), before the gradient pass needs it.
__global__ void __launch_bounds__(1024)
cos_count(const uint8_t *__restrict__ counts, int64_t P, float *__restrict__ out) {
    __shared__ unsigned long long s_n[32];
    unsigned long long n = count_covered(counts, P);
    for (int o = 16; o > 0; o >>= 1) n += __shfl_xor_sync(0xffffffffu, n, o);
    if ((threadIdx.x & 31) == 0) s_n[threadIdx.x >> 5] = n;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long nn = 0;
        for (int w = 0; w < int(blockDim.x >> 5); ++w) nn += s_n[w];
        out[1] = float(1.0 / (nn > 0 ? double(nn) : 1.0));
    }
}

// One warp per pixel: the pixel's term 1 - cos and its gradient row, already
// multiplied by 1/n.  VEC: 16-byte loads and stores (C % 4 == 0, aligned rows).
template <bool VEC>
__global__ void __launch_bounds__(T)
cos_terms(const float *__restrict__ F, const float *__restrict__ tgt,
          const uint8_t *__restrict__ counts, int64_t P, int C, float eps,
          float *__restrict__ term, float *__restrict__ grad, const float *__restrict__ out) {
    const int lane = threadIdx.x & 31;
    const int64_t w0 = (int64_t(blockIdx.x) * T + threadIdx.x) >> 5;
    const int64_t nw = (int64_t(gridDim.x) * T) >> 5;
    const float s = out[1];
    for (int64_t p = w0; p < P; p += nw) {
        const bool on = counts[p] > 0;
        const float *f = F + p * C;
        const float *t = tgt + p * C;
        float dot = 0.f, ff = 0.f, tt = 0.f;
        if (VEC) {
            const float4 *f4 = reinterpret_cast<const float4 *>(f);
            const float4 *t4 = reinterpret_cast<const float4 *>(t);
            for (int c = lane; c < C / 4; c += 32) {
                const float4 a = f4[c], b = t4[c];
                dot = fmaf(a.x, b.x, fmaf(a.y, b.y, fmaf(a.z, b.z, fmaf(a.w, b.w, dot))));
                ff = fmaf(a.x, a.x, fmaf(a.y, a.y, fmaf(a.z, a.z, fmaf(a.w, a.w, ff))));
                tt = fmaf(b.x, b.x, fmaf(b.y, b.y, fmaf(b.z, b.z, fmaf(b.w, b.w, tt))));
            }
        } else {
            for (int c = lane; c < C; c += 32) {
                const float a = f[c], b = t[c];
                dot = fmaf(a, b, dot);
                ff = fmaf(a, a, ff);
                tt = fmaf(b, b, tt);
            }
        }
        for (int o = 16; o > 0; o >>= 1) {
            dot += __shfl_xor_sync(0xffffffffu, dot, o);
            ff += __shfl_xor_sync(0xffffffffu, ff, o);
            tt += __shfl_xor_sync(0xffffffffu, tt, o);
        }
        const float nf_raw = sqrtf(ff), nt = fmaxf(sqrtf(tt), eps);
        const bool big = nf_raw > eps;
        const float nf = big ? nf_raw : eps;
        const float cs = dot / (nf * nt);
        if (lane == 0) term[p] = on ? 1.f - cs : 0.f;
        float *gp = grad + p * C;
        const float k1 = 1.f / (nf * nt), k2 = big ? dot / (nf * nf * nf * nt) : 0.f;
        if (VEC) {
            const float4 *f4 = reinterpret_cast<const float4 *>(f);
            const float4 *t4 = reinterpret_cast<const float4 *>(t);
            float4 *g4 = reinterpret_cast<float4 *>(gp);
            for (int c = lane; c < C / 4; c += 32) {
                if (!on) { g4[c] = make_float4(0.f, 0.f, 0.f, 0.f); continue; }
                const float4 a = f4[c], b = t4[c];
                g4[c] = make_float4(-(b.x * k1 - a.x * k2) * s, -(b.y * k1 - a.y * k2) * s,
                                    -(b.z * k1 - a.z * k2) * s, -(b.w * k1 - a.w * k2) * s);
            }
        } else {
            for (int c = lane; c < C; c += 32) gp[c] = on ? -(t[c] * k1 - f[c] * k2) * s : 0.f;
        }
    }
}

// FP32 sum with its rounding error carried by Knuth's TwoSum (error-free:
// s + e == a + b exactly), so a thread's few hundred terms keep FP64-like
// accuracy without FP64 arithmetic in the loop.
__device__ __forceinline__ void two_sum_acc(float &s, float &c, float x) {
    const float t = s + x;
    const float bp = t - s;
    c += (s - (t - bp)) + (x - bp);
    s = t;
}

// L = (sum of the terms) / n, coalesced reads in a fixed order, eight loads in
// flight per thread; per-thread compensated sums are combined in double.
__global__ void __launch_bounds__(1024)
cos_final(const float *__restrict__ term, const uint8_t *__restrict__ counts, int64_t P,
          float *__restrict__ out) {
    __shared__ double s_sum[32];
    __shared__ unsigned long long s_n[32];
    float sf = 0.f, cf = 0.f;
    const int64_t step = blockDim.x;
    int64_t i = threadIdx.x;
    for (; i + 7 * step < P; i += 8 * step) {
        float t[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) t[u] = term[i + u * step];
#pragma unroll
        for (int u = 0; u < 8; ++u) two_sum_acc(sf, cf, t[u]);
    }
    for (; i < P; i += step) two_sum_acc(sf, cf, term[i]);
    double sum = double(sf) + double(cf);
    unsigned long long n = count_covered(counts, P);
    for (int o = 16; o > 0; o >>= 1) {
        sum += __shfl_xor_sync(0xffffffffu, sum, o);
        n += __shfl_xor_sync(0xffffffffu, n, o);
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) { s_sum[warp] = sum; s_n[warp] = n; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double sm = 0.0;
        unsigned long long nn = 0;
        for (int w = 0; w < int(blockDim.x >> 5); ++w) { sm += s_sum[w]; nn += s_n[w]; }
        out[0] = float(sm / (nn > 0 ? double(nn) : 1.0));
    }
}

}  // namespace

cudaError_t launch_cosine_loss(const float *F, const float *tgt, const uint8_t *counts, int64_t P,
                               int C, float *term, float *out2, float *grad, cudaStream_t s) {
    int dev = 0, sms = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const bool vec = C % 4 == 0 && (reinterpret_cast<uintptr_t>(F) & 15) == 0 &&
                     (reinterpret_cast<uintptr_t>(tgt) & 15) == 0 &&
                     (reinterpret_cast<uintptr_t>(grad) & 15) == 0;
    cos_count<<<1, 1024, 0, s>>>(counts, P, out2);
    if (vec) cos_terms<true><<<sms * 8, T, 0, s>>>(F, tgt, counts, P, C, 1e-8f, term, grad, out2);
    else cos_terms<false><<<sms * 8, T, 0, s>>>(F, tgt, counts, P, C, 1e-8f, term, grad, out2);
    cos_final<<<1, 1024, 0, s>>>(term, counts, P, out2);
    count_launch(3);
    return cudaGetLastError();
}

}  // namespace qr
