// Cosine loss of the differentiation workload (not in the paper, whose loss is
// the contrastive Eq. 2 on CLIP targets): L = mean over pixels with at least
// one quantile Gaussian of 1 - cos(F_p, t_p), cos = F.t / (max(|F|,eps) max(|t|,eps)),
// and its gradient dL/dF.  Deterministic: the covered pixels are counted
// first (integer atomics, so the count does not depend on their order), one
// pass writes every pixel's term and its gradient row already scaled by 1/n,
// and the terms are summed over fixed contiguous ranges, one per CTA, whose
// sums the last CTA to finish adds in a fixed order.  out[0] and out[1] hold
// the ticket and the count as integers until that CTA writes (L, 1/n).
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

// Number of covered pixels, added into out[1] as an integer (zeroed before),
// before the gradient pass needs it.  CTA b counts the pixels of range b:
// [b range, (b + 1) range), the last one up to P.
__global__ void __launch_bounds__(1024)
cos_count(const uint8_t *__restrict__ counts, int64_t P, int64_t range, float *__restrict__ out) {
    __shared__ unsigned long long s_n[32];
    const int64_t i0 = int64_t(blockIdx.x) * range;
    const int64_t len = blockIdx.x + 1 == gridDim.x ? P - i0 : range;   // the last range takes the rest
    unsigned long long n = len > 0 ? count_covered(counts + i0, len) : 0ull;
    for (int o = 16; o > 0; o >>= 1) n += __shfl_xor_sync(0xffffffffu, n, o);
    if ((threadIdx.x & 31) == 0) s_n[threadIdx.x >> 5] = n;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long nn = 0;
        for (int w = 0; w < int(blockDim.x >> 5); ++w) nn += s_n[w];
        if (nn) atomicAdd(reinterpret_cast<unsigned int *>(out + 1), unsigned(nn));
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
    const float s = cos_inv_count(out);
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
        const CosCoeffs cc = cos_coeffs(dot, ff, tt, eps);
        if (lane == 0) term[p] = on ? 1.f - cc.cs : 0.f;
        float *gp = grad + p * C;
        const float k1 = cc.k1, k2 = cc.k2;
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

// L = (sum of the terms) / n.  CTA b sums the terms of range b (coalesced
// reads, eight loads in flight per thread, compensated per-thread sums
// combined in double).  With one CTA it writes L directly; otherwise it
// stores its sum, as the two 32-bit halves of a double, over the first two
// terms of its range (every range holds at least 8192), which no other CTA
// reads, and the last CTA to take a ticket adds the sums in a fixed order
// (lane l of its first warp the sums l, l + 32, ..., then a butterfly).
__global__ void __launch_bounds__(1024)
cos_final(float *__restrict__ term, int64_t P, int64_t range, float *__restrict__ out) {
    __shared__ double s_sum[32];
    __shared__ unsigned s_ticket;
    const int64_t i0 = int64_t(blockIdx.x) * range;
    const int64_t len = blockIdx.x + 1 == gridDim.x ? P - i0 : range;   // the last range takes the rest
    const float *t0 = term + i0;
    float sf = 0.f, cf = 0.f;
    const int64_t step = blockDim.x;
    int64_t i = threadIdx.x;
    for (; i + 7 * step < len; i += 8 * step) {
        float t[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) t[u] = t0[i + u * step];
#pragma unroll
        for (int u = 0; u < 8; ++u) two_sum_acc(sf, cf, t[u]);
    }
    for (; i < len; i += step) two_sum_acc(sf, cf, t0[i]);
    double sum = double(sf) + double(cf);
    for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) s_sum[warp] = sum;
    __syncthreads();   // every read of this range is done
    if (gridDim.x == 1) {
        if (threadIdx.x == 0) {
            double sm = 0.0;
            for (int w = 0; w < int(blockDim.x >> 5); ++w) sm += s_sum[w];
            const unsigned nn = *reinterpret_cast<const volatile unsigned int *>(out + 1);
            const double n = nn > 0 ? double(nn) : 1.0;
            out[0] = float(sm / n);
            out[1] = float(1.0 / n);
        }
        return;
    }
    if (threadIdx.x == 0) {
        double sm = 0.0;
        for (int w = 0; w < int(blockDim.x >> 5); ++w) sm += s_sum[w];
        unsigned *slot = reinterpret_cast<unsigned *>(term + i0);
        slot[0] = unsigned(__double2loint(sm));
        slot[1] = unsigned(__double2hiint(sm));
        __threadfence();
        s_ticket = atomicAdd(reinterpret_cast<unsigned int *>(out), 1u);
    }
    __syncthreads();
    if (s_ticket != gridDim.x - 1 || threadIdx.x >= 32) return;
    __threadfence();
    // the last CTA's first warp: lane l adds the range sums l, l + 32, ... in
    // order, then the lanes' sums meet in a fixed butterfly
    double total = 0.0;
    for (unsigned b = threadIdx.x; b < gridDim.x; b += 32) {
        const volatile unsigned *slot = reinterpret_cast<const volatile unsigned *>(term + int64_t(b) * range);
        total += __hiloint2double(int(slot[1]), int(slot[0]));
    }
    for (int o = 16; o > 0; o >>= 1) total += __shfl_xor_sync(0xffffffffu, total, o);
    if (threadIdx.x != 0) return;
    const unsigned nn = *reinterpret_cast<const volatile unsigned int *>(out + 1);
    const double n = nn > 0 ? double(nn) : 1.0;
    out[0] = float(total / n);
    out[1] = float(1.0 / n);
}

}  // namespace

namespace {
// ranges of at least 8192 pixels (each holds the two words of its sum), at
// most two per SM; the last range takes the rest of the pixels
struct Ranges {
    int64_t range;
    unsigned nblk;
};
Ranges loss_ranges(int64_t P, int sms) {
    int64_t range = (P + 2 * sms - 1) / (2 * sms);
    if (range < 8192) range = 8192;
    return {range, unsigned(P / range > 1 ? P / range : 1)};
}
int sm_count() {
    int dev = 0, sms = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sms;
}
}  // namespace

cudaError_t launch_cos_count(const uint8_t *counts, int64_t P, float *out2, cudaStream_t s) {
    const Ranges r = loss_ranges(P, sm_count());
    cudaError_t e = cudaMemsetAsync(out2, 0, 2 * sizeof(float), s);
    if (e != cudaSuccess) return e;
    cos_count<<<r.nblk, 1024, 0, s>>>(counts, P, r.range, out2);
    count_launch(1);
    return cudaGetLastError();
}

cudaError_t launch_cos_final(float *term, int64_t P, float *out2, cudaStream_t s) {
    const Ranges r = loss_ranges(P, sm_count());
    cos_final<<<r.nblk, 1024, 0, s>>>(term, P, r.range, out2);
    count_launch(1);
    return cudaGetLastError();
}

cudaError_t launch_cosine_loss(const float *F, const float *tgt, const uint8_t *counts, int64_t P,
                               int C, float *term, float *out2, float *grad, cudaStream_t s) {
    const int sms = sm_count();
    const bool vec = C % 4 == 0 && (reinterpret_cast<uintptr_t>(F) & 15) == 0 &&
                     (reinterpret_cast<uintptr_t>(tgt) & 15) == 0 &&
                     (reinterpret_cast<uintptr_t>(grad) & 15) == 0;
    cudaError_t e = launch_cos_count(counts, P, out2, s);
    if (e != cudaSuccess) return e;
    if (vec) cos_terms<true><<<sms * 8, T, 0, s>>>(F, tgt, counts, P, C, 1e-8f, term, grad, out2);
    else cos_terms<false><<<sms * 8, T, 0, s>>>(F, tgt, counts, P, C, 1e-8f, term, grad, out2);
    count_launch(1);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return launch_cos_final(term, P, out2, s);
}

}  // namespace qr
