// The training loss of the paper, Eq. 2 (Sec. 4.3), on a rendered map:
// pixel p lies in mask (patch) i = mask_id[p] whose CLIP embedding is t_i;
// with s_j = cos(F_p, t_j) = F.t_j / (max(|F|,eps) max(|t_j|,eps)),
//     L_p = -log( exp(s_i) / sum_{j != i} exp(s_j) ) = -s_i + log sum_{j != i} exp(s_j)
// (the denominator over the other masks, as Eq. 2 prints it), and L is the
// mean over the pixels with mask_id >= 0 (count floored at 1).  Its gradient:
//     dL_p/dF = (1/n) [ sum_j c_j t^_j / nf - (sum_j c_j s_j) F / nf^2 ],
// c_i = -1, c_j = exp(s_j) / sum_{l != i} exp(s_l), t^_j = t_j / max(|t_j|, eps),
// nf = max(|F|, eps) (no second term where |F| <= eps).
//
// GB300 design: the pass is two contractions with the M unit targets (the
// similarities F T^T and the gradient C T), P x C x M multiply-adds each.
//   * eq2_norm writes the unit targets t^ (one warp per target) and
//     eq2_count counts the pixels in the loss (integer atomics), ahead of the
//     pass that needs 1/n;
//   * eq2_terms: one persistent CTA per SM holds all M unit targets in shared
//     memory (M x C FP32); each warp takes four pixels at a time with their
//     feature rows in registers (a lane owns 4 x C/128 channels of each), so
//     every target slice read from shared memory feeds four pixels.  Partial
//     dot products of 16 targets are reduced across the lanes by a halving
//     butterfly (31 shuffles per pixel for 16 targets instead of 80), the
//     softmax over the other masks runs one target per lane, and the
//     gradient rows are accumulated from the same shared targets and written
//     once, already scaled by 1/n, with the pixel's loss term;
//   * the terms are summed by the cosine loss's deterministic range sums.
// FP32 throughout (exp and log with the accurate expf / logf), so the loss
// and its gradient meet an FP64 reference to a few units of FP32 rounding.
#include "qr_internal.cuh"

namespace qr {
namespace {

constexpr int kThreads = 256;
constexpr int kPB = 4;          // pixels per warp at a time
constexpr int kTB = 16;         // targets per reduction block

__global__ void eq2_norm(const float *__restrict__ tgt, int M, int C, float eps,
                         float *__restrict__ tn) {
    const int lane = threadIdx.x & 31;
    const int j = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (j >= M) return;
    const float *t = tgt + int64_t(j) * C;
    float ss = 0.f;
    for (int c = lane; c < C; c += 32) ss = fmaf(t[c], t[c], ss);
    for (int o = 16; o > 0; o >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, o);
    const float inv = 1.0f / fmaxf(sqrtf(ss), eps);
    for (int c = lane; c < C; c += 32) tn[int64_t(j) * C + c] = t[c] * inv;
}

// pixels with mask_id >= 0, added into out[1] as an integer (zeroed before)
__global__ void __launch_bounds__(1024)
eq2_count(const int32_t *__restrict__ mask_id, int64_t P, float *__restrict__ out) {
    __shared__ unsigned s_n[32];
    unsigned n = 0;
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < P;
         i += int64_t(gridDim.x) * blockDim.x)
        n += mask_id[i] >= 0;
    for (int o = 16; o > 0; o >>= 1) n += __shfl_xor_sync(0xffffffffu, n, o);
    if ((threadIdx.x & 31) == 0) s_n[threadIdx.x >> 5] = n;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned nn = 0;
        for (int w = 0; w < int(blockDim.x >> 5); ++w) nn += s_n[w];
        if (nn) atomicAdd(reinterpret_cast<unsigned int *>(out + 1), nn);
    }
}

// Halving butterfly: on entry each lane holds kTB partial sums v[0..kTB);
// on exit lane l holds the full sum of entry (l & (kTB-1)) (lanes l and l ^ 16
// hold the same).
__device__ __forceinline__ float reduce_block16(float (&v)[kTB], int lane) {
    constexpr unsigned FULL = 0xffffffffu;
#pragma unroll
    for (int i = 0; i < kTB; ++i) v[i] += __shfl_xor_sync(FULL, v[i], 16);
#pragma unroll
    for (int half = kTB / 2; half >= 1; half >>= 1) {
        const bool up = (lane & half) != 0;
#pragma unroll
        for (int i = 0; i < half; ++i) {
            const float keep = up ? v[i + half] : v[i];
            const float send = up ? v[i] : v[i + half];
            v[i] = keep + __shfl_xor_sync(FULL, send, half);
        }
    }
    return v[0];
}

// VPL float4 per lane per row (C = 128 VPL)
template <int VPL>
__global__ void __launch_bounds__(kThreads, 1)
eq2_terms(const float *__restrict__ F, const float *__restrict__ tn, int M, int C,
          const int32_t *__restrict__ mask_id, int64_t P, float eps, float *__restrict__ term,
          float *__restrict__ grad, const float *__restrict__ out2) {
    constexpr unsigned FULL = 0xffffffffu;
    constexpr int NW = kThreads / 32;
    extern __shared__ __align__(16) float s_t[];          // [M][C] unit targets
    __shared__ float s_sc[NW][kPB][64];                  // per warp: similarities, then c_j
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int i = threadIdx.x; i < M * C / 4; i += kThreads)
        reinterpret_cast<float4 *>(s_t)[i] = reinterpret_cast<const float4 *>(tn)[i];
    __syncthreads();
    const float inv_n = cos_inv_count(out2);
    const int64_t groups = (P + kPB - 1) / kPB;
    for (int64_t gi = int64_t(blockIdx.x) * NW + warp; gi < groups; gi += int64_t(gridDim.x) * NW) {
        const int64_t p0 = gi * kPB;
        float fr[kPB][VPL * 4];
        float nf[kPB], nfr[kPB];
        int mid[kPB];
#pragma unroll
        for (int p = 0; p < kPB; ++p) {
            const bool ok = p0 + p < P;
            mid[p] = ok ? mask_id[p0 + p] : -1;
            float ff = 0.f;
#pragma unroll
            for (int v = 0; v < VPL; ++v) {
                const float4 x = ok ? reinterpret_cast<const float4 *>(F + (p0 + p) * int64_t(C))[lane + 32 * v]
                                    : make_float4(0.f, 0.f, 0.f, 0.f);
                fr[p][4 * v] = x.x; fr[p][4 * v + 1] = x.y; fr[p][4 * v + 2] = x.z; fr[p][4 * v + 3] = x.w;
                ff = fmaf(x.x, x.x, fmaf(x.y, x.y, fmaf(x.z, x.z, fmaf(x.w, x.w, ff))));
            }
            for (int o = 16; o > 0; o >>= 1) ff += __shfl_xor_sync(FULL, ff, o);
            nfr[p] = sqrtf(ff);
            nf[p] = fmaxf(nfr[p], eps);
        }
        // similarities s_j = F . t^_j / nf, 16 targets at a time
        for (int j0 = 0; j0 < M; j0 += kTB) {
            float part[kPB][kTB];
#pragma unroll
            for (int p = 0; p < kPB; ++p)
#pragma unroll
                for (int jj = 0; jj < kTB; ++jj) part[p][jj] = 0.f;
#pragma unroll
            for (int jj = 0; jj < kTB; ++jj) {
                const int j = j0 + jj < M ? j0 + jj : M - 1;
                const float4 *tr = reinterpret_cast<const float4 *>(s_t + int64_t(j) * C);
#pragma unroll
                for (int v = 0; v < VPL; ++v) {
                    const float4 t = tr[lane + 32 * v];
#pragma unroll
                    for (int p = 0; p < kPB; ++p) {
                        part[p][jj] = fmaf(fr[p][4 * v], t.x, part[p][jj]);
                        part[p][jj] = fmaf(fr[p][4 * v + 1], t.y, part[p][jj]);
                        part[p][jj] = fmaf(fr[p][4 * v + 2], t.z, part[p][jj]);
                        part[p][jj] = fmaf(fr[p][4 * v + 3], t.w, part[p][jj]);
                    }
                }
            }
#pragma unroll
            for (int p = 0; p < kPB; ++p) {
                const float d = reduce_block16(part[p], lane);
                const int j = j0 + (lane & (kTB - 1));
                if (lane < kTB && j < M) s_sc[warp][p][j] = d / nf[p];
            }
        }
        __syncwarp();
        // softmax over the other masks: one target per lane (M <= 64)
        float cs[kPB];
#pragma unroll
        for (int p = 0; p < kPB; ++p) {
            const int i = mid[p];
            const float si = i >= 0 ? s_sc[warp][p][i] : 0.f;
            float e[2], sj[2];
            float Z = 0.f;
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int j = lane + 32 * h;
                sj[h] = j < M ? s_sc[warp][p][j] : 0.f;
                e[h] = (j < M && j != i) ? expf(sj[h]) : 0.f;
                Z += e[h];
            }
            for (int o = 16; o > 0; o >>= 1) Z += __shfl_xor_sync(FULL, Z, o);
            __syncwarp();   // every lane has read the similarities before they are replaced
            float csum = 0.f;
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int j = lane + 32 * h;
                const float c = j == i ? -1.f : e[h] / Z;
                csum = fmaf(c, sj[h], csum);
                if (j < M) s_sc[warp][p][j] = i >= 0 ? c * inv_n : 0.f;
            }
            for (int o = 16; o > 0; o >>= 1) csum += __shfl_xor_sync(FULL, csum, o);
            cs[p] = csum;
            if (lane == 0 && p0 + p < P) term[p0 + p] = i >= 0 ? logf(Z) - si : 0.f;
        }
        __syncwarp();
        // gradient rows: (sum_j c_j t^_j) / nf - (sum_j c_j s_j) F / nf^2, times 1/n
        float acc[kPB][VPL * 4];
#pragma unroll
        for (int p = 0; p < kPB; ++p)
#pragma unroll
            for (int q = 0; q < VPL * 4; ++q) acc[p][q] = 0.f;
        for (int j = 0; j < M; ++j) {
            const float4 *tr = reinterpret_cast<const float4 *>(s_t + int64_t(j) * C);
            float cj[kPB];
#pragma unroll
            for (int p = 0; p < kPB; ++p) cj[p] = s_sc[warp][p][j];
#pragma unroll
            for (int v = 0; v < VPL; ++v) {
                const float4 t = tr[lane + 32 * v];
#pragma unroll
                for (int p = 0; p < kPB; ++p) {
                    acc[p][4 * v] = fmaf(cj[p], t.x, acc[p][4 * v]);
                    acc[p][4 * v + 1] = fmaf(cj[p], t.y, acc[p][4 * v + 1]);
                    acc[p][4 * v + 2] = fmaf(cj[p], t.z, acc[p][4 * v + 2]);
                    acc[p][4 * v + 3] = fmaf(cj[p], t.w, acc[p][4 * v + 3]);
                }
            }
        }
#pragma unroll
        for (int p = 0; p < kPB; ++p) {
            if (p0 + p >= P) break;
            const bool on = mid[p] >= 0;
            const float a1 = 1.0f / nf[p];
            const float a2 = nfr[p] > eps ? cs[p] * inv_n / (nf[p] * nf[p]) : 0.f;
            float4 *g = reinterpret_cast<float4 *>(grad + (p0 + p) * int64_t(C));
#pragma unroll
            for (int v = 0; v < VPL; ++v) {
                float4 o;
                o.x = on ? fmaf(acc[p][4 * v], a1, -a2 * fr[p][4 * v]) : 0.f;
                o.y = on ? fmaf(acc[p][4 * v + 1], a1, -a2 * fr[p][4 * v + 1]) : 0.f;
                o.z = on ? fmaf(acc[p][4 * v + 2], a1, -a2 * fr[p][4 * v + 2]) : 0.f;
                o.w = on ? fmaf(acc[p][4 * v + 3], a1, -a2 * fr[p][4 * v + 3]) : 0.f;
                __stcg(g + lane + 32 * v, o);
            }
        }
        __syncwarp();   // s_sc is rewritten by the next group
    }
}

int sm_count_now() {
    int dev = 0, sms = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sms;
}

}  // namespace

bool contrastive_supported(int M, int C) {
    return M >= 2 && M <= 64 && C % 128 == 0 && C >= 128 && C <= 512 &&
           size_t(M) * C * 4 <= 200 * 1024;
}

size_t contrastive_workspace_bytes(int64_t P, int M, int C) {
    return ((size_t(M) * C * 4 + 255) & ~size_t(255)) + ((size_t(P) * 4 + 255) & ~size_t(255));
}

cudaError_t launch_contrastive_loss(const float *F, const float *tgt, int M, int C,
                                    const int32_t *mask_id, int64_t P, float *out2, float *grad,
                                    void *ws, cudaStream_t s) {
    float *tn = static_cast<float *>(ws);
    float *term = reinterpret_cast<float *>(static_cast<char *>(ws) +
                                            ((size_t(M) * C * 4 + 255) & ~size_t(255)));
    const int sms = sm_count_now();
    cudaError_t e = cudaMemsetAsync(out2, 0, 2 * sizeof(float), s);
    if (e != cudaSuccess) return e;
    eq2_norm<<<(M * 32 + 255) / 256, 256, 0, s>>>(tgt, M, C, 1e-8f, tn);
    eq2_count<<<unsigned(sms), 1024, 0, s>>>(mask_id, P, out2);
    const size_t dyn = size_t(M) * C * 4;
    auto go = [&](auto kern) -> cudaError_t {
        cudaError_t ee = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(dyn));
        if (ee != cudaSuccess) return ee;
        kern<<<unsigned(sms), kThreads, dyn, s>>>(F, tn, M, C, mask_id, P, 1e-8f, term, grad, out2);
        return cudaGetLastError();
    };
    switch (C / 128) {
        case 1: e = go(eq2_terms<1>); break;
        case 2: e = go(eq2_terms<2>); break;
        case 3: e = go(eq2_terms<3>); break;
        default: e = go(eq2_terms<4>); break;
    }
    count_launch(3);
    if (e != cudaSuccess) return e;
    return launch_cos_final(term, P, out2, s);
}

}  // namespace qr
