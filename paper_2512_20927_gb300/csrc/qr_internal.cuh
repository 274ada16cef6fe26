// Internal declarations shared by the libqrender translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/qrender.h"

namespace qr {

// Programmatic dependent launch: a kernel launched by pdl_launch may be
// scheduled while its predecessor on the stream is still finishing, so its
// launch overlaps the predecessor's last blocks; its first statement is
// pdl_wait(), which returns once the predecessor has completed and its writes
// are visible (a no-op for a kernel launched without the attribute).
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

template <typename... KArgs, typename... Args>
inline cudaError_t pdl_launch(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem,
                              cudaStream_t s, Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, args...);
}

// ---------------------------------------------------------------- status word
// counters[0]: device status (a qr_status value, 0 = OK)
// counters[1]: number of tile-Gaussian intersections the frame needs
// counters[2]: number of kept Gaussians (non-empty footprint)
// counters[3]: number of Gaussians n
// counters[4]: number of intersections actually emitted (0 on overflow)
enum { CNT_STATUS = 0, CNT_ISECT = 1, CNT_VISIBLE = 2, CNT_N = 3, CNT_SORT_N = 4, CNT_CAND = 5,
       CNT_BIG = 6, CNT_WORDS = 8 };

// Workspace slots (byte offsets in qr_frame::off).
enum Slot {
    S_COUNTERS = 0, S_DIFF, S_REC_M, S_REC_C, S_REC_A, S_REC_H, S_RECT, S_TCOUNT, S_GKEY,
    S_VISCNT, S_BSUM, S_KID, S_OFF, S_TCNT, S_RANGES, S_KEYS64, S_SCRATCH64, S_IGID,
    S_CHUNK,
    S_END
};
constexpr int kProjectThreads = 256;
// Copies of the 2-D difference array of per-tile counts; CTA b adds into copy
// b % kDiffCopies, which spreads the atomics on its hot corners.  S_DIFF
// follows S_COUNTERS so that one memset clears both.
constexpr int kDiffCopies = 8;
// Output slots per expansion chunk (the binning records the owner of each
// chunk's first slot).
constexpr int kEmitChunk = 1024;
static_assert(S_END <= QR_FRAME_SLOTS, "too many workspace slots");

constexpr int kKMax = 32;

// Launch counter (all TUs add to it).
void count_launch(int n = 1);

template <typename T>
__host__ __device__ inline T *slot(void *ws, const qr_frame &f, Slot s) {
    return reinterpret_cast<T *>(static_cast<char *>(ws) + f.off[s]);
}
template <typename T>
inline T *slot(const qr_frame &f, Slot s) {
    return reinterpret_cast<T *>(static_cast<char *>(f.ws) + f.off[s]);
}

inline int64_t num_pixels(const qr_frame &f) {
    return int64_t(f.camera.width) * int64_t(f.camera.height);
}
inline int32_t num_tiles(const qr_frame &f) { return f.tiles_x * f.tiles_y; }

// ---------------------------------------------------------------- launchers
cudaError_t launch_project(const qr_frame &f, const float *mean, const float *log_scale,
                           const float *quat, const float *opacity, cudaStream_t s);
cudaError_t launch_sort(const qr_frame &f, cudaStream_t s);
cudaError_t launch_select(const qr_frame &f, int32_t *ids, float *w, uint8_t *cnt, bool riemann,
                          cudaStream_t s);
// stats (nullable, wide rows only): [0] += blended (pixel, Gaussian) pairs,
// [1] += executed (8-pixel group, entry) pairs of the accumulation
cudaError_t launch_dense(const qr_frame &f, const void *feat, const float *scale, qr_dtype dt,
                         int C, float *out, float *T_final, cudaStream_t s,
                         unsigned long long *stats = nullptr);
// rule: 1 = top-K, 2 = Stratified-K (qr_rule); tau [P][K] nullable (stratified boundaries)
cudaError_t launch_select_rule(const qr_frame &f, int rule, int32_t *ids, float *w, uint8_t *cnt,
                               float *tau, cudaStream_t s);

size_t backward_workspace_bytes(const qr_frame &f, int C);
cudaError_t launch_backward(const qr_frame &f, const void *feat, const float *scale, qr_dtype dt,
                            int C, const int32_t *ids, const float *w, const uint8_t *cnt,
                            const float *grad_out, float *grad_feat, float *grad_alpha,
                            float *grad_conic, void *ws, cudaStream_t s);
cudaError_t launch_cosine_loss(const float *F, const float *tgt, const uint8_t *counts, int64_t P,
                               int C, float *term, float *out2, float *grad, cudaStream_t s);
// the loss's two reductions, for a caller that forms the terms and the
// gradient itself: the covered-pixel count into out2[1] (zeroed first) and
// the final in-order sum that leaves (L, 1/n) in out2
cudaError_t launch_cos_count(const uint8_t *counts, int64_t P, float *out2, cudaStream_t s);
cudaError_t launch_cos_final(float *term, int64_t P, float *out2, cudaStream_t s);

// The cosine loss fused into the backward's per-pixel pass: F, tgt [P][C],
// mask [P] (pixels in the loss), term [P] scratch, out2 [2] -> (L, 1/n),
// grad_map [P][C] -> dL/dF (then the backward's upstream gradient).
struct CosLossArgs {
    const float *F;
    const float *tgt;
    const uint8_t *mask;
    float *term;
    float *out2;
    float *grad_map;
};
size_t backward_cos_workspace_bytes(const qr_frame &f, int C);   // + P floats of loss terms
cudaError_t launch_backward_cos(const qr_frame &f, const void *feat, const float *scale,
                                qr_dtype dt, int C, const int32_t *ids, const float *w,
                                const uint8_t *cnt, const CosLossArgs &loss, float *grad_feat,
                                float *grad_alpha, float *grad_conic, void *ws, cudaStream_t s);

// 1/n from the integer covered-pixel count that out2[1] holds between the
// count and the final sum
__device__ __forceinline__ float cos_inv_count(const float *out2) {
    const unsigned nn = *reinterpret_cast<const volatile unsigned int *>(out2 + 1);
    return float(1.0 / (nn > 0 ? double(nn) : 1.0));
}

// Per-pixel cosine term from the reduced dot = F.t, ff = |F|^2, tt = |t|^2:
// cs = F.t / (max(|F|,eps) max(|t|,eps)); dL/dF = -(t k1 - F k2) / n with
// k1 = 1 / (nf nt) and k2 = F.t / (nf^3 nt) (zero when |F| <= eps, where
// max(|F|, eps) is constant).
struct CosCoeffs {
    float cs, k1, k2;
};
__device__ __forceinline__ CosCoeffs cos_coeffs(float dot, float ff, float tt, float eps) {
    const float nf_raw = sqrtf(ff), nt = fmaxf(sqrtf(tt), eps);
    const bool big = nf_raw > eps;
    const float nf = big ? nf_raw : eps;
    CosCoeffs c;
    c.cs = dot / (nf * nt);
    c.k1 = 1.f / (nf * nt);
    c.k2 = big ? dot / (nf * nf * nf * nt) : 0.f;
    return c;
}

struct BatchView;
bool batch_supported(qr_dtype dt, int C);
bool batch_chunks_ok(int C, int chunks);
size_t batch_desc_bytes(int n_views);
size_t batch_view_size();
cudaError_t launch_batch(const void *ws, int n_views, uint32_t total_items, qr_dtype dt, int C,
                         int K, int group, int chunks, int blend_warps, int ctas_per_sm,
                         cudaStream_t s);
cudaError_t prepare_batch(const qr_view *views, int n_views, void *ws, uint32_t *total_items,
                          cudaStream_t s, BatchView *host_scratch);
// Eq. 2 contrastive loss (contrastive.cu): out2 -> (L, 1/n), grad [P][C] -> dL/dF;
// ws: contrastive_workspace_bytes (unit targets, per-pixel terms)
bool contrastive_supported(int M, int C);
size_t contrastive_workspace_bytes(int64_t P, int M, int C);
cudaError_t launch_contrastive_loss(const float *F, const float *tgt, int M, int C,
                                    const int32_t *mask_id, int64_t P, float *out2, float *grad,
                                    void *ws, cudaStream_t s);
bool relevance_supported(int Q, int C);
void set_wait_limit(unsigned polls);
bool set_blend_chunks(int chunks);
// blend of qr_blend fused with the relevance product (the map is never written)
bool blend_relevance_supported(qr_dtype dt, int Q, int C, int K);
cudaError_t launch_blend_relevance(const void *feat, const float *scale, qr_dtype dt, int C,
                                   int64_t n_gauss, const int32_t *ids, const float *w,
                                   const uint8_t *cnt, int64_t P, int K, int W, int H,
                                   const uint16_t *q, int Q, float *out, int *status,
                                   cudaStream_t s);
cudaError_t launch_relevance(const float *map, const uint16_t *q, int Q, int64_t P, int C,
                             float *out, int *status, cudaStream_t s);



// ---------------------------------------------------------------- block scans
// Inclusive scan of one value per thread across the CTA (blockDim.x a
// multiple of 32, at most 1024); returns the inclusive prefix and the total.
__device__ __forceinline__ uint32_t block_inclusive_scan(uint32_t v, uint32_t *s_w, uint32_t &total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) s_w[warp] = x;
    __syncthreads();
    if (warp == 0) {
        uint32_t w = (lane < nw) ? s_w[lane] : 0u;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        s_w[lane] = w;
    }
    __syncthreads();
    const uint32_t r = x + (warp > 0 ? s_w[warp - 1] : 0u);
    total = s_w[nw - 1];
    __syncthreads();
    return r;
}

// Exclusive scan of `total` u32 in place by one CTA: coalesced chunks of
// blockDim.x elements with a running carry.  Returns the grand total to
// thread 0 through *sum_out (nullable).
__device__ __forceinline__ void cta_exclusive_scan(uint32_t *data, int total, uint32_t *sum_out) {
    __shared__ uint32_t s_w[32];
    uint32_t carry = 0;
    for (int base = 0; base < total; base += blockDim.x) {
        const int i = base + threadIdx.x;
        const uint32_t v = i < total ? data[i] : 0u;
        uint32_t chunk;
        const uint32_t inc = block_inclusive_scan(v, s_w, chunk);
        if (i < total) data[i] = carry + inc - v;
        carry += chunk;
    }
    if (sum_out && threadIdx.x == 0) *sum_out = carry;
}

// Two independent inclusive scans in one pass (x and y of one uint2 per
// thread); s_w holds 64 words.
__device__ __forceinline__ uint2 block_inclusive_scan2(uint2 v, uint32_t *s_w, uint2 &total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    uint2 x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t a = __shfl_up_sync(0xffffffffu, x.x, o);
        const uint32_t b = __shfl_up_sync(0xffffffffu, x.y, o);
        if (lane >= o) { x.x += a; x.y += b; }
    }
    if (lane == 31) { s_w[warp] = x.x; s_w[32 + warp] = x.y; }
    __syncthreads();
    if (warp == 0) {
        uint32_t a = (lane < nw) ? s_w[lane] : 0u, b = (lane < nw) ? s_w[32 + lane] : 0u;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t ya = __shfl_up_sync(0xffffffffu, a, o);
            const uint32_t yb = __shfl_up_sync(0xffffffffu, b, o);
            if (lane >= o) { a += ya; b += yb; }
        }
        s_w[lane] = a;
        s_w[32 + lane] = b;
    }
    __syncthreads();
    const uint2 r = make_uint2(x.x + (warp > 0 ? s_w[warp - 1] : 0u), x.y + (warp > 0 ? s_w[32 + warp - 1] : 0u));
    total = make_uint2(s_w[nw - 1], s_w[32 + nw - 1]);
    __syncthreads();
    return r;
}

// ---------------------------------------------------------------- per-pixel Gaussian
// Every kernel evaluates alpha' at a pixel the same way.  The projected
// Gaussian is stored as its mean (hi + lo) and two scaled principal axes
// w1, w2 of the conic, A = 2 (w1 w1^T + w2 w2^T), so that
//     q/2 = (d . w1)^2 + (d . w2)^2,   d = u - mu'.
// The sum of squares has no cancellation (the conic form
// A00 dx^2 + 2 A01 dx dy + A11 dy^2 loses up to cond(Sigma') ulps for
// elongated Gaussians), and costs five FP32 operations.
struct PixelTerm {
    float dx, dy, half_q;
};
__device__ __forceinline__ PixelTerm eval_half_q(float ux, float uy, float4 m, float4 w) {
    PixelTerm t;
    t.dx = (ux - m.x) - m.z;
    t.dy = (uy - m.y) - m.w;
    const float p1 = fmaf(t.dx, w.x, t.dy * w.y);
    const float p2 = fmaf(t.dx, w.z, t.dy * w.w);
    t.half_q = fmaf(p1, p1, p2 * p2);
    return t;
}
__device__ __forceinline__ float eval_alpha(float alpha, float half_q, float alpha_max) {
    return fminf(alpha_max, alpha * __expf(-half_q));
}
// A pixel whose q/2 exceeds this bound cannot reach alpha' >= alpha_min:
// alpha exp(-q/2) < alpha_min exactly when q/2 > ln(alpha / alpha_min); the 1 %
// + 0.01 margin is far above the FP32 error of q/2 and of the exponential, so
// skipping these pixels before the exponential changes no decision.
__device__ __forceinline__ float reject_half_q(float alpha, float alpha_min) {
    return fmaf(logf(fmaxf(alpha / alpha_min, 1.0f)), 1.01f, 0.01f);
}

// Lower end of q/2 = (d.w1)^2 + (d.w2)^2, d = u - mu', over the box
// [x0,x1] x [y0,y1] of pixel centres: 0 if mu' is inside, else the smallest
// value on the four edges, each at its clamped 1-D minimiser (evaluated with
// the same dot products as a pixel, so no cancellation-prone closed form).
__device__ __forceinline__ float box_min_half_q(float4 mm, float4 cc, float x0, float x1, float y0,
                                                float y1) {
    const float mx = mm.x + mm.z, my = mm.y + mm.w;
    if (mx >= x0 && mx <= x1 && my >= y0 && my <= y1) return 0.0f;
    const float sxy = fmaf(cc.x, cc.y, cc.z * cc.w);
    const float sxx = fmaf(cc.x, cc.x, cc.z * cc.z), syy = fmaf(cc.y, cc.y, cc.w * cc.w);
    // the edge minimisers only choose where q/2 is evaluated, so an approximate
    // quotient suffices (inf / NaN clamp to an edge end)
    const float ky = -__fdividef(sxy, syy), kx = -__fdividef(sxy, sxx);
    float best = INFINITY;
#pragma unroll
    for (int e = 0; e < 2; ++e) {
        const float dx = (e ? x1 : x0) - mx;
        const float dy = fminf(fmaxf(dx * ky, y0 - my), y1 - my);
        const float p1 = fmaf(dx, cc.x, dy * cc.y), p2 = fmaf(dx, cc.z, dy * cc.w);
        best = fminf(best, fmaf(p1, p1, p2 * p2));
    }
#pragma unroll
    for (int e = 0; e < 2; ++e) {
        const float dy = (e ? y1 : y0) - my;
        const float dx = fminf(fmaxf(dy * kx, x0 - mx), x1 - mx);
        const float p1 = fmaf(dx, cc.x, dy * cc.y), p2 = fmaf(dx, cc.z, dy * cc.w);
        best = fminf(best, fmaf(p1, p1, p2 * p2));
    }
    return best;
}

// ---------------------------------------------------------------- Algorithm 1 walk
// Algorithm 1 state of one pixel.
struct Walk {
    float T, TQ, thr;
    int k, m;
    bool done;
};

// The rarely taken end of an Algorithm 1 step, for a member entry (alpha' >=
// alpha_min) whose T_test = Tt crosses the next quantile boundary or the stop
// threshold: keep the Gaussian, advance k, stop.  The kept weight is
// T^Q alpha' (Algorithm 1), or with kCount the number of boundaries Tt
// crosses (App. C's right-Riemann weights, one segment width per boundary).
template <bool kCount = false>
__device__ __forceinline__ void walk_event(Walk &w, float Tt, float a, float tau_stop, int K,
                                        uint32_t gid, int slot, int KS, int32_t *s_ids, float *s_w) {
    if (Tt < w.thr) {
        const int k0 = w.k;
        s_ids[slot * KS + w.m] = int32_t(gid);
        if constexpr (!kCount) s_w[slot * KS + w.m] = w.TQ * a;
        ++w.m;
        w.TQ = w.TQ * (1.0f - a);
        do {
            ++w.k;
            w.thr = (w.k < K) ? __fdiv_rn(float(K - w.k), float(K + 1)) : -1.0f;
        } while (Tt < w.thr);
        if constexpr (kCount) s_w[slot * KS + w.m - 1] = float(w.k - k0);
    }
    if (Tt < tau_stop) w.done = true;
    else w.T = Tt;
}

// ---------------------------------------------------------------- register bitonic sort
// Sorts NTH*E keys (32- or 64-bit) held E per thread in blocked order (thread t holds
// positions tE .. tE+E-1; pad with ~0).  Compare-exchange partners i and i^j
// meet inside a thread for j < E (register swaps), across lanes for
// E <= j < 32E (shuffles) and across warps for larger j (the shared-memory
// buffer s of NTH*E keys, two barriers per stage).  All NTH threads call it.
__device__ __forceinline__ unsigned long long shfl_xor_key(unsigned long long x, int m) {
    const uint32_t lo = __shfl_xor_sync(0xffffffffu, uint32_t(x), m);
    const uint32_t hi = __shfl_xor_sync(0xffffffffu, uint32_t(x >> 32), m);
    return (static_cast<unsigned long long>(hi) << 32) | lo;
}
__device__ __forceinline__ uint32_t shfl_xor_key(uint32_t x, int m) {
    return __shfl_xor_sync(0xffffffffu, x, m);
}

// The smaller of (a, b) when take_min, else the larger.
template <typename KT>
__device__ __forceinline__ KT key_pick(KT a, KT b, bool take_min) {
    return ((a < b) == take_min) ? a : b;
}

// Position i = base + e of a thread's keys differs from base only below bit
// log2(E) (base is a multiple of E), so for strides j >= E and blocks k > j
// the direction of a compare-exchange is the same for all E keys of a thread
// and is computed once per stage.
template <int E, int NTH, typename KT>
__device__ void bitonic_regs(KT (&v)[E], KT *s) {
    constexpr int N = NTH * E;
    const int base = threadIdx.x * E;
    for (int k = 2; k <= N; k <<= 1) {
        const bool up = (base & k) == 0;
        for (int j = k >> 1; j >= 32 * E; j >>= 1) {
            // exchange through s element-major (key e of thread t at e NTH + t):
            // a warp's accesses are consecutive words, free of bank conflicts
#pragma unroll
            for (int e = 0; e < E; ++e) s[e * NTH + threadIdx.x] = v[e];
            __syncthreads();
            const bool take_min = ((base & j) == 0) == up;
            const KT *partner = s + (threadIdx.x ^ (j / E));
#pragma unroll
            for (int e = 0; e < E; ++e) v[e] = key_pick(v[e], partner[e * NTH], take_min);
            __syncthreads();
        }
        for (int j = min(k >> 1, 16 * E); j >= E; j >>= 1) {
            const bool take_min = ((base & j) == 0) == up;
#pragma unroll
            for (int e = 0; e < E; ++e) v[e] = key_pick(v[e], shfl_xor_key(v[e], j / E), take_min);
        }
#pragma unroll
        for (int J = E / 2; J > 0; J >>= 1) {
            if (J >= k) continue;
#pragma unroll
            for (int e = 0; e < E; ++e) {
                if ((e ^ J) > e) {
                    const bool u = k >= E ? up : ((e & k) == 0);
                    const KT a = v[e], b = v[e ^ J];
                    if ((a > b) == u) { v[e] = b; v[e ^ J] = a; }
                }
            }
        }
    }
}

// ---------------------------------------------------------------- compensated arithmetic
// Pairs (hi, lo) of FP32 with |lo| <= ulp(hi)/2 represent hi + lo exactly;
// the error-free transformations are Knuth's TwoSum, Dekker's FastTwoSum and
// the FMA-based TwoProduct; division is Dekker's long division with two
// correction steps.  Explicit _rn intrinsics keep nvcc from contracting or
// reassociating them.
struct df {
    float hi, lo;
};

__device__ __forceinline__ df df_two_sum(float a, float b) {
    float s = __fadd_rn(a, b);
    float bb = __fsub_rn(s, a);
    float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return {s, e};
}
__device__ __forceinline__ df df_fast_two_sum(float a, float b) {  // needs |a| >= |b| or a == 0
    float s = __fadd_rn(a, b);
    float e = __fsub_rn(b, __fsub_rn(s, a));
    return {s, e};
}
__device__ __forceinline__ df df_two_prod(float a, float b) {
    float p = __fmul_rn(a, b);
    float e = __fmaf_rn(a, b, -p);
    return {p, e};
}
__device__ __forceinline__ df df_from(float a) { return {a, 0.0f}; }
__device__ __forceinline__ df df_neg(df a) { return {-a.hi, -a.lo}; }
__device__ __forceinline__ df df_add(df a, df b) {
    df s = df_two_sum(a.hi, b.hi);
    df t = df_two_sum(a.lo, b.lo);
    s.lo = __fadd_rn(s.lo, t.hi);
    s = df_fast_two_sum(s.hi, s.lo);
    s.lo = __fadd_rn(s.lo, t.lo);
    return df_fast_two_sum(s.hi, s.lo);
}
__device__ __forceinline__ df df_sub(df a, df b) { return df_add(a, df_neg(b)); }
__device__ __forceinline__ df df_add_f(df a, float b) {
    df s = df_two_sum(a.hi, b);
    s.lo = __fadd_rn(s.lo, a.lo);
    return df_fast_two_sum(s.hi, s.lo);
}
__device__ __forceinline__ df df_mul(df a, df b) {
    df p = df_two_prod(a.hi, b.hi);
    p.lo = __fmaf_rn(a.hi, b.lo, p.lo);
    p.lo = __fmaf_rn(a.lo, b.hi, p.lo);
    return df_fast_two_sum(p.hi, p.lo);
}
__device__ __forceinline__ df df_mul_f(df a, float b) {
    df p = df_two_prod(a.hi, b);
    p.lo = __fmaf_rn(a.lo, b, p.lo);
    return df_fast_two_sum(p.hi, p.lo);
}
__device__ __forceinline__ df df_div(df a, df b) {
    float q1 = __fdiv_rn(a.hi, b.hi);
    df r = df_sub(a, df_mul_f(b, q1));
    float q2 = __fdiv_rn(r.hi, b.hi);
    r = df_sub(r, df_mul_f(b, q2));
    float q3 = __fdiv_rn(r.hi, b.hi);
    df q = df_fast_two_sum(q1, q2);
    return df_add_f(q, q3);
}
// Square root with one Newton correction of the FP32 estimate.
__device__ __forceinline__ df df_sqrt(df a) {
    if (!(a.hi > 0.f)) return {0.f, 0.f};
    const float s = sqrtf(a.hi);
    const df r = df_sub(a, df_two_prod(s, s));
    return df_fast_two_sum(s, __fdiv_rn(r.hi, 2.0f * s));
}
__device__ __forceinline__ float df_abs_hi(df a) { return fabsf(a.hi); }
// a*b + c*d + e*f, all in df.
__device__ __forceinline__ df df_dot3(df a, df b, df c, df d, df e, df f) {
    return df_add(df_add(df_mul(a, b), df_mul(c, d)), df_mul(e, f));
}

}  // namespace qr
