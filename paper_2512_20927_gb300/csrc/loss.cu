// Cosine loss of the differentiation workload (not in the paper, whose loss is
// the contrastive Eq. 2 on CLIP targets): L = mean over pixels with at least
// one quantile Gaussian of 1 - cos(F_p, t_p), cos = F.t / (max(|F|,eps) max(|t|,eps)),
// and its gradient dL/dF.  Deterministic: per-pixel terms, then one CTA sums
// them in a fixed order.
#include "qr_internal.cuh"

namespace qr {
namespace {

constexpr int T = 256;

__global__ void __launch_bounds__(T)
cos_terms(const float *__restrict__ F, const float *__restrict__ tgt,
          const uint8_t *__restrict__ counts, int64_t P, int C, float eps,
          float *__restrict__ term, float *__restrict__ grad) {
    const int lane = threadIdx.x & 31;
    const int64_t w0 = (int64_t(blockIdx.x) * T + threadIdx.x) >> 5;
    const int64_t nw = (int64_t(gridDim.x) * T) >> 5;
    for (int64_t p = w0; p < P; p += nw) {
        const bool on = counts[p] > 0;
        const float *f = F + p * C;
        const float *t = tgt + p * C;
        float dot = 0.f, ff = 0.f, tt = 0.f;
        for (int c = lane; c < C; c += 32) {
            const float a = f[c], b = t[c];
            dot = fmaf(a, b, dot);
            ff = fmaf(a, a, ff);
            tt = fmaf(b, b, tt);
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
        for (int c = lane; c < C; c += 32) gp[c] = on ? -(t[c] * k1 - f[c] * k2) : 0.f;
    }
}

__global__ void __launch_bounds__(1024)
cos_reduce(const float *__restrict__ term, const uint8_t *__restrict__ counts, int64_t P,
           float *__restrict__ out /* [loss, 1/n] */) {
    __shared__ double s_sum[32];
    __shared__ unsigned long long s_n[32];
    double sum = 0.0;
    unsigned long long n = 0;
    const int64_t per = (P + blockDim.x - 1) / blockDim.x;
    const int64_t a = min(P, int64_t(threadIdx.x) * per), b = min(P, a + per);
    for (int64_t i = a; i < b; ++i) {
        sum += double(term[i]);
        n += counts[i] > 0;
    }
    for (int o = 16; o > 0; o >>= 1) {
        sum += __shfl_xor_sync(0xffffffffu, sum, o);
        n += __shfl_xor_sync(0xffffffffu, n, o);
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) { s_sum[warp] = sum; s_n[warp] = n; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        unsigned long long nn = 0;
        for (int w = 0; w < int(blockDim.x >> 5); ++w) { s += s_sum[w]; nn += s_n[w]; }
        const double d = nn > 0 ? double(nn) : 1.0;
        out[0] = float(s / d);
        out[1] = float(1.0 / d);
    }
}

__global__ void __launch_bounds__(T)
scale_grad(float *__restrict__ grad, int64_t count, const float *__restrict__ out) {
    const float s = out[1];
    for (int64_t i = int64_t(blockIdx.x) * T + threadIdx.x; i < count; i += int64_t(gridDim.x) * T)
        grad[i] *= s;
}

}  // namespace

cudaError_t launch_cosine_loss(const float *F, const float *tgt, const uint8_t *counts, int64_t P,
                               int C, float *term, float *out2, float *grad, cudaStream_t s) {
    int dev = 0, sms = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cos_terms<<<sms * 8, T, 0, s>>>(F, tgt, counts, P, C, 1e-8f, term, grad);
    cos_reduce<<<1, 1024, 0, s>>>(term, counts, P, out2);
    scale_grad<<<sms * 8, T, 0, s>>>(grad, P * int64_t(C), out2);
    count_launch(3);
    return cudaGetLastError();
}

}  // namespace qr
