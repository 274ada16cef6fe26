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
//   * up to 32 targets, eq2_mma: both
//     contractions on the tensor cores as 3xTF32 mma.sync products (the
//     operands split into TF32 hi and lo parts, hi*hi + hi*lo + lo*hi with
//     FP32 accumulation, which keeps FP32 accuracy), described at the kernel;
//   * otherwise eq2_terms: one persistent CTA per SM holds all M unit targets in shared
//     memory (M x C FP32); each warp takes four pixels at a time with their
//     feature rows in registers (a lane owns 4 x C/128 channels of each), so
//     every target slice read from shared memory feeds four pixels.  Partial
//     dot products of 16 targets are reduced across the lanes by a halving
//     butterfly (31 shuffles per pixel for 16 targets instead of 80), the
//     softmax over the other masks runs one target per lane, and the
//     gradient rows are accumulated from the same shared targets and written
//     once, already scaled by 1/n, with the pixel's loss term;
//   * the terms are summed by the cosine loss's deterministic range sums.
// FP32 arithmetic (exp and log with the accurate expf / logf; the 3xTF32
// products carry about FP32 precision), so the loss and its gradient meet an
// FP64 reference to a few units of FP32 rounding.
#include "qr_internal.cuh"
#include "mma_tf32.cuh"

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

// ------------------------------------------------------------------ tensor cores
// The two contractions on the tensor cores in the 3xTF32 form of
// mma_tf32.cuh (mma.sync m16n8k8, FP32-class accuracy).

// eq2_mma: M <= 16 MT targets.  One CTA per SM holds the unit targets split
// into TF32 hi / lo parts in shared memory ([16 MT][C + 16] each; the row pad
// makes the fragment loads conflict-free); each warp takes 16 pixels at a
// time (two 8-pixel n-tiles; g = lane / 4, t = lane % 4):
//   1. S^T = T^ F^T (M = targets, N = pixels, K = channels): per 16
//      channels a lane loads one float4 of each of its two pixel rows, the
//      next 32 channels' loads in flight meanwhile (the
//      K order inside the 16 is permuted so that A and B fragments are float4
//      loads; the sums are the same) and accumulates |F|^2;
//   2. per pixel, from the accumulator layout (lane (g, t) holds targets g,
//      g + 8 of each 16 for pixels 2t, 2t + 1 of each n-tile): s_j, the
//      softmax over the other masks, the loss term and c_j, with reductions
//      over the eight lanes that share t;
//   3. G = C T^ (M = pixels, N = channels, K = targets): the c_j fragments
//      are gathered by shuffles, T^ fragments read from shared memory, and
//      each 16 x 8 result, (G / nf - (sum_j c_j s_j) F / nf^2) / n, is
//      written (streaming stores) with the F values it needs re-read (they
//      were read moments before and come from L2).
constexpr int kMmaThreads = 512;

template <int MT>
__global__ void __launch_bounds__(kMmaThreads, 1)
eq2_mma(const float *__restrict__ F, const float *__restrict__ tn, int M, int C,
        const int32_t *__restrict__ mask_id, int64_t P, float eps, float *__restrict__ term,
        float *__restrict__ grad, const float *__restrict__ out2) {
    constexpr unsigned FULL = 0xffffffffu;
    constexpr int NW = kMmaThreads / 32;
    constexpr int NT = 2;                  // 8-pixel n-tiles per warp
    constexpr int NPX = 8 * NT;            // pixels per warp block
    constexpr int MR = 16 * MT;            // target rows held
    extern __shared__ __align__(16) float s_t[];
    const int S = C + 16;
    float *s_hi = s_t, *s_lo = s_t + MR * S;
    __shared__ float s_a1[NW][NPX], s_a2[NW][NPX];
    for (int i = threadIdx.x; i < MR * C; i += kMmaThreads) {
        const int j = i / C, c = i - j * C;
        const float x = j < M ? tn[int64_t(j) * C + c] : 0.f;
        uint32_t h, l;
        split_tf32(x, h, l);
        s_hi[j * S + c] = __uint_as_float(h);
        s_lo[j * S + c] = __uint_as_float(l);
    }
    __syncthreads();
    const float inv_n = cos_inv_count(out2);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int g = lane >> 2, t = lane & 3;
    const int64_t blocks = (P + NPX - 1) / NPX;
    for (int64_t blk = int64_t(blockIdx.x) * NW + warp; blk < blocks; blk += int64_t(gridDim.x) * NW) {
        const int64_t p0 = blk * NPX;
        // ---------------- 1. similarities
        float acc[MT][NT][4];
        float ff[NT];
#pragma unroll
        for (int nt = 0; nt < NT; ++nt) {
            ff[nt] = 0.f;
#pragma unroll
            for (int mt = 0; mt < MT; ++mt)
#pragma unroll
                for (int q = 0; q < 4; ++q) acc[mt][nt][q] = 0.f;
        }
        // the next 16 channels' F values are loaded while the current ones are used
        float4 fq[NT];
        auto load_f = [&](int cg, float4 (&dst)[NT]) {
#pragma unroll
            for (int nt = 0; nt < NT; ++nt) {
                const int64_t px = p0 + nt * 8 + g;
                dst[nt] = (px < P && cg < C)
                              ? __ldg(reinterpret_cast<const float4 *>(F + px * C + cg + 4 * t))
                              : make_float4(0.f, 0.f, 0.f, 0.f);
            }
        };
        float4 fn[NT];
        load_f(0, fq);
        load_f(16, fn);
        for (int cg = 0; cg < C; cg += 16) {
            float4 fn2[NT];
            load_f(cg + 32, fn2);   // two groups of loads in flight ahead of the MMAs
            // A fragments of every m-tile (rows g and g + 8, channels cg + 4t ..):
            // k-step 0 takes .x (slot t) and .y (slot t + 4), k-step 1 .z and .w
            uint32_t ah[MT][2][4], al[MT][2][4];
#pragma unroll
            for (int mt = 0; mt < MT; ++mt) {
                const float4 h0 = *reinterpret_cast<const float4 *>(s_hi + (16 * mt + g) * S + cg + 4 * t);
                const float4 h1 = *reinterpret_cast<const float4 *>(s_hi + (16 * mt + g + 8) * S + cg + 4 * t);
                const float4 l0 = *reinterpret_cast<const float4 *>(s_lo + (16 * mt + g) * S + cg + 4 * t);
                const float4 l1 = *reinterpret_cast<const float4 *>(s_lo + (16 * mt + g + 8) * S + cg + 4 * t);
                ah[mt][0][0] = __float_as_uint(h0.x); ah[mt][0][1] = __float_as_uint(h1.x);
                ah[mt][0][2] = __float_as_uint(h0.y); ah[mt][0][3] = __float_as_uint(h1.y);
                ah[mt][1][0] = __float_as_uint(h0.z); ah[mt][1][1] = __float_as_uint(h1.z);
                ah[mt][1][2] = __float_as_uint(h0.w); ah[mt][1][3] = __float_as_uint(h1.w);
                al[mt][0][0] = __float_as_uint(l0.x); al[mt][0][1] = __float_as_uint(l1.x);
                al[mt][0][2] = __float_as_uint(l0.y); al[mt][0][3] = __float_as_uint(l1.y);
                al[mt][1][0] = __float_as_uint(l0.z); al[mt][1][1] = __float_as_uint(l1.z);
                al[mt][1][2] = __float_as_uint(l0.w); al[mt][1][3] = __float_as_uint(l1.w);
            }
#pragma unroll
            for (int nt = 0; nt < NT; ++nt) {
                const float4 x = fq[nt];
                ff[nt] = fmaf(x.x, x.x, fmaf(x.y, x.y, fmaf(x.z, x.z, fmaf(x.w, x.w, ff[nt]))));
                uint32_t bh[4], bl[4];
                split_tf32(x.x, bh[0], bl[0]);
                split_tf32(x.y, bh[1], bl[1]);
                split_tf32(x.z, bh[2], bl[2]);
                split_tf32(x.w, bh[3], bl[3]);
#pragma unroll
                for (int mt = 0; mt < MT; ++mt) {
                    mma3(acc[mt][nt], ah[mt][0], al[mt][0], bh[0], bh[1], bl[0], bl[1]);
                    mma3(acc[mt][nt], ah[mt][1], al[mt][1], bh[2], bh[3], bl[2], bl[3]);
                }
            }
#pragma unroll
            for (int nt = 0; nt < NT; ++nt) {
                fq[nt] = fn[nt];
                fn[nt] = fn2[nt];
            }
        }
#pragma unroll
        for (int nt = 0; nt < NT; ++nt) {
            ff[nt] += __shfl_xor_sync(FULL, ff[nt], 1);
            ff[nt] += __shfl_xor_sync(FULL, ff[nt], 2);
        }
        // ---------------- 2. softmax over the other masks, loss terms, c_j
        // lane (g, t) holds, for pixel nt*8 + 2t + b, targets 16 mt + g + 8 h
        // in acc[mt][nt][2 h + b]; the eight lanes sharing t hold all targets
#pragma unroll
        for (int nt = 0; nt < NT; ++nt) {
#pragma unroll
            for (int b = 0; b < 2; ++b) {
                const int pl = nt * 8 + 2 * t + b;
                const int64_t px = p0 + pl;
                const float nfr = sqrtf(__shfl_sync(FULL, ff[nt], (2 * t + b) * 4));
                const float nf = fmaxf(nfr, eps);
                const int i = px < P ? mask_id[px] : -1;
                float e[MT][2], sv[MT][2];
                float Z = 0.f, si = 0.f;
#pragma unroll
                for (int mt = 0; mt < MT; ++mt)
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        const int j = 16 * mt + g + 8 * h;
                        sv[mt][h] = acc[mt][nt][2 * h + b] / nf;
                        e[mt][h] = (j < M && j != i) ? expf(sv[mt][h]) : 0.f;
                        Z += e[mt][h];
                        if (j == i) si += sv[mt][h];
                    }
#pragma unroll
                for (int o = 4; o < 32; o <<= 1) {
                    Z += __shfl_xor_sync(FULL, Z, o);
                    si += __shfl_xor_sync(FULL, si, o);
                }
                float cs = 0.f;
#pragma unroll
                for (int mt = 0; mt < MT; ++mt)
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        const int j = 16 * mt + g + 8 * h;
                        const float c = j >= M ? 0.f : (j == i ? -1.f : e[mt][h] / Z);
                        cs = fmaf(c, sv[mt][h], cs);
                        acc[mt][nt][2 * h + b] = i >= 0 ? c * inv_n : 0.f;
                    }
#pragma unroll
                for (int o = 4; o < 32; o <<= 1) cs += __shfl_xor_sync(FULL, cs, o);
                if (g == 0) {
                    if (px < P) term[px] = i >= 0 ? logf(Z) - si : 0.f;
                    s_a1[warp][pl] = i >= 0 ? 1.0f / nf : 0.f;
                    s_a2[warp][pl] = (i >= 0 && nfr > eps) ? cs * inv_n / (nf * nf) : 0.f;
                }
            }
        }
        __syncwarp();
        // ---------------- 3. gradient rows, 16 pixels x 8 channels at a time
#pragma unroll
        for (int m2 = 0; m2 < NT / 2; ++m2) {
            const int n0 = 2 * m2, n1 = 2 * m2 + 1;     // n-tiles of rows g and g + 8
            uint32_t ch[2 * MT][4], cl[2 * MT][4];
#pragma unroll
            for (int kk = 0; kk < 2 * MT; ++kk) {
                const int mt = kk >> 1, h = kk & 1;
                const int sa = t * 4 + (g >> 1), sb = (t + 4) * 4 + (g >> 1);
                float v[4];
                {
                    const float x0 = __shfl_sync(FULL, acc[mt][n0][2 * h], sa);
                    const float x1 = __shfl_sync(FULL, acc[mt][n0][2 * h + 1], sa);
                    v[0] = (g & 1) ? x1 : x0;                       // (pixel g, target 8kk + t)
                    const float y0 = __shfl_sync(FULL, acc[mt][n1][2 * h], sa);
                    const float y1 = __shfl_sync(FULL, acc[mt][n1][2 * h + 1], sa);
                    v[1] = (g & 1) ? y1 : y0;                       // (pixel g + 8, target 8kk + t)
                    const float z0 = __shfl_sync(FULL, acc[mt][n0][2 * h], sb);
                    const float z1 = __shfl_sync(FULL, acc[mt][n0][2 * h + 1], sb);
                    v[2] = (g & 1) ? z1 : z0;                       // (pixel g, target 8kk + t + 4)
                    const float w0 = __shfl_sync(FULL, acc[mt][n1][2 * h], sb);
                    const float w1 = __shfl_sync(FULL, acc[mt][n1][2 * h + 1], sb);
                    v[3] = (g & 1) ? w1 : w0;                       // (pixel g + 8, target 8kk + t + 4)
                }
#pragma unroll
                for (int q = 0; q < 4; ++q) split_tf32(v[q], ch[kk][q], cl[kk][q]);
            }
            const int pa = 16 * m2 + g, pb = pa + 8;
            const int64_t pxa = p0 + pa, pxb = p0 + pb;
            const float a1a = s_a1[warp][pa], a2a = s_a2[warp][pa];
            const float a1b = s_a1[warp][pb], a2b = s_a2[warp][pb];
            // F values of the F term, one 8-channel step ahead
            auto load_f2 = [&](int64_t px, int c) {
                return (px < P && c < C) ? __ldg(reinterpret_cast<const float2 *>(F + px * C + c))
                                         : make_float2(0.f, 0.f);
            };
            float2 fa = load_f2(pxa, 2 * t), fb = load_f2(pxb, 2 * t);
            for (int c0 = 0; c0 < C; c0 += 8) {
                const float2 fa_n = load_f2(pxa, c0 + 8 + 2 * t), fb_n = load_f2(pxb, c0 + 8 + 2 * t);
                float d[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
                for (int kk = 0; kk < 2 * MT; ++kk) {
                    const int r0 = (8 * kk + t) * S + c0 + g, r1 = r0 + 4 * S;
                    mma3(d, ch[kk], cl[kk], __float_as_uint(s_hi[r0]), __float_as_uint(s_hi[r1]),
                         __float_as_uint(s_lo[r0]), __float_as_uint(s_lo[r1]));
                }
                const int cc = c0 + 2 * t;
                if (pxa < P)
                    __stcs(reinterpret_cast<float2 *>(grad + pxa * C + cc),
                           a1a > 0.f ? make_float2(fmaf(d[0], a1a, -a2a * fa.x), fmaf(d[1], a1a, -a2a * fa.y))
                                     : make_float2(0.f, 0.f));
                if (pxb < P)
                    __stcs(reinterpret_cast<float2 *>(grad + pxb * C + cc),
                           a1b > 0.f ? make_float2(fmaf(d[2], a1b, -a2b * fb.x), fmaf(d[3], a1b, -a2b * fb.y))
                                     : make_float2(0.f, 0.f));
                fa = fa_n;
                fb = fb_n;
            }
        }
        __syncwarp();   // s_a1 / s_a2 are rewritten by the next block
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
    auto go = [&](auto kern, size_t dyn, int nthreads) -> cudaError_t {
        cudaError_t ee = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(dyn));
        if (ee != cudaSuccess) return ee;
        kern<<<unsigned(sms), nthreads, dyn, s>>>(F, tn, M, C, mask_id, P, 1e-8f, term, grad, out2);
        return cudaGetLastError();
    };
    if (M <= 32) {
        // tensor cores: the unit targets split into TF32 hi / lo rows of C + 16
        const size_t dyn2 = size_t(2) * (M <= 16 ? 16 : 32) * size_t(C + 16) * 4;
        e = M <= 16 ? go(eq2_mma<1>, dyn2, kMmaThreads) : go(eq2_mma<2>, dyn2, kMmaThreads);
    } else {
        const size_t dyn = size_t(M) * C * 4;
        switch (C / 128) {
            case 1: e = go(eq2_terms<1>, dyn, kThreads); break;
            case 2: e = go(eq2_terms<2>, dyn, kThreads); break;
            case 3: e = go(eq2_terms<3>, dyn, kThreads); break;
            default: e = go(eq2_terms<4>, dyn, kThreads); break;
        }
    }
    count_launch(3);
    if (e != cudaSuccess) return e;
    return launch_cos_final(term, P, out2, s);
}

}  // namespace qr
