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
// GB300 design: one CTA per screen tile (256 pixels), 128 threads, each
// walking two vertically adjacent pixels of the same column.  The tile's list
// is staged through shared memory 256 entries at a time (gid, projected mean
// hi/lo, conic axes, opacity, reject bound: 44 B each) with coalesced loads;
// the walk reads the staged entries as broadcasts.  The two pixels share the
// x offset, and their y offsets, axis projections and q/2 are computed with
// packed FP32x2 instructions (each half rounds exactly like the scalar
// instruction), so the common case -- an entry out of reach of both pixels,
// four of five entries walked -- costs one shared-memory read set and a
// handful of instructions for two pixels; four entries are evaluated per
// step (independent chains, so a long walk is not one serial latency chain)
// and the ids of the next batch are fetched while the current one is walked.
// Entries within reach take the Algorithm 1 step for both pixels at once (one
// exp per pixel-entry pair, T_test packed), in list order; only keeping a
// Gaussian or stopping branches off.  A CTA stops loading as soon as all of
// its pixels have stopped (__syncthreads_count).
// Kept (id, weight) pairs go to per-pixel shared-memory slots [K][256] so no
// dynamically indexed register array spills, then are written out once.
#include "qr_internal.cuh"

namespace qr {
namespace {

constexpr int kPix = 256;       // pixels per tile
constexpr int kThreads = 128;   // two pixels per thread

__device__ __forceinline__ float2 add2(float2 a, float2 b) {
    float2 d;
    asm("{\n .reg .b64 x, y;\n mov.b64 x, {%2, %3};\n mov.b64 y, {%4, %5};\n"
        " add.rn.f32x2 x, x, y;\n mov.b64 {%0, %1}, x;\n}\n"
        : "=f"(d.x), "=f"(d.y) : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return d;
}
__device__ __forceinline__ float2 mul2(float2 a, float2 b) {
    float2 d;
    asm("{\n .reg .b64 x, y;\n mov.b64 x, {%2, %3};\n mov.b64 y, {%4, %5};\n"
        " mul.rn.f32x2 x, x, y;\n mov.b64 {%0, %1}, x;\n}\n"
        : "=f"(d.x), "=f"(d.y) : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return d;
}
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) {
    float2 d;
    asm("{\n .reg .b64 x, y, z;\n mov.b64 x, {%2, %3};\n mov.b64 y, {%4, %5};\n"
        " mov.b64 z, {%6, %7};\n fma.rn.f32x2 x, x, y, z;\n mov.b64 {%0, %1}, x;\n}\n"
        : "=f"(d.x), "=f"(d.y)
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y), "f"(c.x), "f"(c.y));
    return d;
}

// Algorithm 1 state of one pixel.
struct Walk {
    float T, TQ, thr;
    int k, m;
    bool done;
};

// The rarely taken end of an Algorithm 1 step, for a member entry (alpha' >=
// alpha_min) whose T_test = Tt crosses the next quantile boundary or the stop
// threshold: keep the Gaussian, advance k, stop.
__device__ __forceinline__ void walk_event(Walk &w, float Tt, float a, float tau_stop, int K,
                                        uint32_t gid, int slot, int32_t *s_ids, float *s_w) {
    if (Tt < w.thr) {
        s_ids[w.m * kPix + slot] = int32_t(gid);
        s_w[w.m * kPix + slot] = w.TQ * a;
        ++w.m;
        w.TQ = w.TQ * (1.0f - a);
        do {
            ++w.k;
            w.thr = (w.k < K) ? __fdiv_rn(float(K - w.k), float(K + 1)) : -1.0f;
        } while (Tt < w.thr);
    }
    if (Tt < tau_stop) w.done = true;
    else w.T = Tt;
}

__global__ void __launch_bounds__(kThreads)
select_kernel(const float4 *__restrict__ rec_m, const float4 *__restrict__ rec_w,
              const float *__restrict__ rec_a, const float *__restrict__ rec_h,
              const uint32_t *__restrict__ isect_gid, const uint2 *__restrict__ ranges, int W,
              int H, int tile_w, int tiles_x, int K, float alpha_min, float alpha_max,
              int32_t *__restrict__ ids, float *__restrict__ wout, uint8_t *__restrict__ cnt) {
    __shared__ float4 s_m[kPix];
    __shared__ float4 s_c[kPix];
    __shared__ float s_a[kPix];
    __shared__ float s_h[kPix];
    __shared__ uint32_t s_g[kPix];
    extern __shared__ unsigned char s_dyn[];
    int32_t *s_ids = reinterpret_cast<int32_t *>(s_dyn);          // [K][256]
    float *s_w = reinterpret_cast<float *>(s_dyn) + K * kPix;     // [K][256]

    const int tile = blockIdx.x;
    const int tx = tile % tiles_x, ty = tile / tiles_x;
    const int tile_h = kPix / tile_w;
    const int lx = threadIdx.x % tile_w, ly = 2 * (threadIdx.x / tile_w);
    const int px = tx * tile_w + lx, py = ty * tile_h + ly;
    const int slot0 = ly * tile_w + lx, slot1 = slot0 + tile_w;
    const bool in0 = px < W && py < H, in1 = px < W && py + 1 < H;
    const float ux = float(px) + 0.5f;
    const float2 uy = make_float2(float(py) + 0.5f, float(py + 1) + 0.5f);
    const uint2 range = ranges[tile];

    const float tau_stop = __fdiv_rn(1.0f, float(K + 1));
    const float thr0 = __fdiv_rn(float(K), float(K + 1));
    Walk w0{1.0f, 1.0f, thr0, 0, 0, !in0};
    Walk w1{1.0f, 1.0f, thr0, 0, 0, !in1};

    // ids of the next batch are fetched while the current batch is walked
    uint32_t gnext[kPix / kThreads];
#pragma unroll
    for (int u = 0; u < kPix / kThreads; ++u) {
        const uint32_t idx = range.x + threadIdx.x + u * kThreads;
        gnext[u] = idx < range.y ? isect_gid[idx] : 0u;
    }
    for (uint32_t b = range.x; b < range.y; b += kPix) {
        if (__syncthreads_count(w0.done && w1.done) == kThreads) break;
#pragma unroll
        for (int u = 0; u < kPix / kThreads; ++u) {
            const int e = threadIdx.x + u * kThreads;
            if (b + e < range.y) {
                const uint32_t g = gnext[u];
                s_g[e] = g;
                s_m[e] = rec_m[g];
                s_c[e] = rec_w[g];
                s_a[e] = rec_a[g];
                s_h[e] = rec_h[g];
            }
        }
        __syncthreads();
#pragma unroll
        for (int u = 0; u < kPix / kThreads; ++u) {
            const uint32_t idx = b + kPix + threadIdx.x + u * kThreads;
            gnext[u] = idx < range.y ? isect_gid[idx] : 0u;
        }
        const int nb = int(min(uint32_t(kPix), range.y - b));
        if (w0.done && w1.done) continue;
        // four entries per step: their q/2 chains are independent, and the
        // scalar Algorithm 1 steps run only when one of them is within reach
        for (int j0 = 0; j0 < nb; j0 += 4) {
            float2 hq[4];
            float h[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int j = min(j0 + u, nb - 1);
                const float4 mm = s_m[j];
                const float4 cc = s_c[j];
                h[u] = s_h[j];
                // eval_half_q for both pixels: dx shared, the rest packed
                const float dx = (ux - mm.x) - mm.z;
                const float2 dy = add2(add2(uy, make_float2(-mm.y, -mm.y)), make_float2(-mm.w, -mm.w));
                const float2 dx2 = make_float2(dx, dx);
                const float2 p1 = fma2(dx2, make_float2(cc.x, cc.x), mul2(dy, make_float2(cc.y, cc.y)));
                const float2 p2 = fma2(dx2, make_float2(cc.z, cc.z), mul2(dy, make_float2(cc.w, cc.w)));
                hq[u] = fma2(p1, p1, mul2(p2, p2));
            }
            unsigned reach = 0;   // bit 2u: pixel 0 may take entry u, bit 2u+1: pixel 1
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const bool valid = j0 + u < nb;
                reach |= unsigned(valid && !(hq[u].x > h[u])) << (2 * u);
                reach |= unsigned(valid && !(hq[u].y > h[u])) << (2 * u + 1);
            }
            if (w0.done) reach &= 0xAAu;
            if (w1.done) reach &= 0x55u;
            if (!reach) continue;
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const bool r0 = !w0.done && ((reach >> (2 * u)) & 1u);
                const bool r1 = !w1.done && ((reach >> (2 * u + 1)) & 1u);
                if (!(r0 || r1)) continue;
                // alpha' and T_test for both pixels; a pixel for which the entry is
                // not a member gets alpha' = 0, i.e. T_test = T (1 - 0) = T exactly
                const float alpha = s_a[j0 + u];
                const float a0 = eval_alpha(alpha, hq[u].x, alpha_max);
                const float a1 = eval_alpha(alpha, hq[u].y, alpha_max);
                const bool t0 = r0 && !(a0 < alpha_min), t1 = r1 && !(a1 < alpha_min);
                const float2 Tt = mul2(make_float2(w0.T, w1.T),
                                       add2(make_float2(1.0f, 1.0f),
                                            make_float2(t0 ? -a0 : -0.0f, t1 ? -a1 : -0.0f)));
                const bool e0 = t0 && (Tt.x < w0.thr || Tt.x < tau_stop);
                const bool e1 = t1 && (Tt.y < w1.thr || Tt.y < tau_stop);
                if (e0 || e1) {
                    const uint32_t gid = s_g[j0 + u];
                    if (e0) walk_event(w0, Tt.x, a0, tau_stop, K, gid, slot0, s_ids, s_w);
                    if (e1) walk_event(w1, Tt.y, a1, tau_stop, K, gid, slot1, s_ids, s_w);
                }
                if (t0 && !e0) w0.T = Tt.x;
                if (t1 && !e1) w1.T = Tt.y;
            }
            if (w0.done && w1.done) break;
        }
    }
    const float D0 = 1.0f - w0.TQ, D1 = 1.0f - w1.TQ;
    for (int j = 0; j < K; ++j) {
        if (in0) {
            const int64_t p = int64_t(py) * W + px;
            const bool has = j < w0.m;
            ids[p * K + j] = has ? s_ids[j * kPix + slot0] : -1;
            wout[p * K + j] = has ? __fdiv_rn(s_w[j * kPix + slot0], D0) : 0.0f;
        }
        if (in1) {
            const int64_t p = int64_t(py + 1) * W + px;
            const bool has = j < w1.m;
            ids[p * K + j] = has ? s_ids[j * kPix + slot1] : -1;
            wout[p * K + j] = has ? __fdiv_rn(s_w[j * kPix + slot1], D1) : 0.0f;
        }
    }
    if (in0) cnt[int64_t(py) * W + px] = uint8_t(w0.m);
    if (in1) cnt[int64_t(py + 1) * W + px] = uint8_t(w1.m);
}

}  // namespace

cudaError_t launch_select(const qr_frame &f, int32_t *ids, float *w, uint8_t *cnt,
                          cudaStream_t s) {
    const int tiles = num_tiles(f);
    if (tiles == 0) return cudaSuccess;
    const int K = f.params.K;
    const size_t dyn = size_t(K) * kPix * 8;
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
