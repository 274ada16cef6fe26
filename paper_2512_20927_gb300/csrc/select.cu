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
// the ids of the next batch are fetched while the current one is walked.
//   * Each warp first culls the staged entries against its box of pixel
//     centres (16x4 for 16x16 tiles), one entry per lane: the minimum of q/2
//     over the box against the entry's reject bound.  About four of five
//     entries a pixel would walk are out of reach of the whole box; the
//     survivors form a per-warp list in shared memory, in list order.
//   * The warp walks its list four entries per step (independent chains).
//     The two pixels of a thread share the x offset; their y offsets, axis
//     projections and q/2 use packed FP32x2 instructions (each half rounds
//     exactly like the scalar instruction).  Entries within reach take the
//     Algorithm 1 step for both pixels at once (one exp per pixel-entry pair,
//     T_test packed); only keeping a Gaussian or stopping branches off.
// A CTA stops loading as soon as all of its pixels have stopped
// (__syncthreads_count).  Kept (id, weight) pairs go to per-pixel
// shared-memory slots [256][K|1] (no dynamically indexed register array, no
// bank conflicts) and are written out once per tile row as contiguous runs of
// tile_w * K ids and weights, so the stores are fully coalesced.
#include "qr_internal.cuh"

namespace qr {
namespace {

constexpr int kPix = 256;       // pixels per tile
constexpr int kThreads = 128;   // two pixels per thread
constexpr int kBatch = 128;     // list entries staged per batch

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

__global__ void __launch_bounds__(kThreads, 8)
select_kernel(const float4 *__restrict__ rec_m, const float4 *__restrict__ rec_w,
              const float *__restrict__ rec_a, const float *__restrict__ rec_h,
              const uint32_t *__restrict__ isect_gid, const uint2 *__restrict__ ranges, int W,
              int H, int tile_w, int tiles_x, int K, float alpha_min, float alpha_max,
              int32_t *__restrict__ ids, float *__restrict__ wout, uint8_t *__restrict__ cnt) {
    pdl_wait();   // the predecessor's outputs are complete and visible
    __shared__ float4 s_m[kBatch];
    __shared__ float4 s_c[kBatch];
    __shared__ float s_a[kBatch];
    __shared__ float s_h[kBatch];
    __shared__ uint32_t s_g[kBatch];
    __shared__ float s_D[kPix];       // 1 - T^Q per pixel
    __shared__ uint8_t s_cnt[kPix];
    extern __shared__ unsigned char s_dyn[];
    const int KS = K | 1;   // odd stride: the per-pixel slots fall in distinct banks
    int32_t *s_ids = reinterpret_cast<int32_t *>(s_dyn);          // [256][KS]
    float *s_w = reinterpret_cast<float *>(s_dyn) + KS * kPix;    // [256][KS]

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

    // the warp's box of pixel centres
    constexpr unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    float bx0 = ux, bx1 = ux, by0 = uy.x, by1 = uy.y;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        bx0 = fminf(bx0, __shfl_xor_sync(FULL, bx0, o));
        bx1 = fmaxf(bx1, __shfl_xor_sync(FULL, bx1, o));
        by0 = fminf(by0, __shfl_xor_sync(FULL, by0, o));
        by1 = fmaxf(by1, __shfl_xor_sync(FULL, by1, o));
    }

    // the id of the next staged entry is fetched while the current batch is walked
    uint32_t gnext = range.x + threadIdx.x < range.y ? isect_gid[range.x + threadIdx.x] : 0u;
    for (uint32_t b = range.x; b < range.y; b += kBatch) {
        if (__syncthreads_count(w0.done && w1.done) == kThreads) break;
        if (b + threadIdx.x < range.y) {
            s_g[threadIdx.x] = gnext;
            s_m[threadIdx.x] = rec_m[gnext];
            s_c[threadIdx.x] = rec_w[gnext];
            s_a[threadIdx.x] = rec_a[gnext];
            s_h[threadIdx.x] = rec_h[gnext];
        }
        __syncthreads();
        {
            const uint32_t idx = b + kBatch + threadIdx.x;
            gnext = idx < range.y ? isect_gid[idx] : 0u;
        }
        const int nb = int(min(uint32_t(kBatch), range.y - b));
        for (int c0 = 0; c0 < nb; c0 += 32) {
            if (__all_sync(FULL, w0.done && w1.done)) break;
            // cull 32 staged entries against the warp's box (one per lane): an
            // entry whose q/2 stays above its reject bound over the whole box
            // is skipped by every pixel of the warp anyway
            const int jl = c0 + lane;
            bool pass = false;
            if (jl < nb)
                pass = !(box_min_half_q(s_m[jl], s_c[jl], bx0, bx1, by0, by1) * 0.999f > s_h[jl] + 1e-3f);
            unsigned todo = __ballot_sync(FULL, pass);
            // walk the survivors in list order, four entries per step: their
            // q/2 chains are independent, and the Algorithm 1 steps run only
            // when one of them is within reach
            while (todo) {
                int jj[4];
                bool valid[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    valid[u] = todo != 0u;
                    jj[u] = valid[u] ? c0 + __ffs(todo) - 1 : jj[0];
                    todo &= todo - 1u;
                }
                float2 hq[4];
                float h[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int j = jj[u];
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
                    reach |= unsigned(valid[u] && !(hq[u].x > h[u])) << (2 * u);
                    reach |= unsigned(valid[u] && !(hq[u].y > h[u])) << (2 * u + 1);
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
                    const float alpha = s_a[jj[u]];
                    const float a0 = eval_alpha(alpha, hq[u].x, alpha_max);
                    const float a1 = eval_alpha(alpha, hq[u].y, alpha_max);
                    const bool t0 = r0 && !(a0 < alpha_min), t1 = r1 && !(a1 < alpha_min);
                    const float2 Tt = mul2(make_float2(w0.T, w1.T),
                                           add2(make_float2(1.0f, 1.0f),
                                                make_float2(t0 ? -a0 : -0.0f, t1 ? -a1 : -0.0f)));
                    const bool e0 = t0 && (Tt.x < w0.thr || Tt.x < tau_stop);
                    const bool e1 = t1 && (Tt.y < w1.thr || Tt.y < tau_stop);
                    if (e0 || e1) {
                        const uint32_t gid = s_g[jj[u]];
                        if (e0) walk_event(w0, Tt.x, a0, tau_stop, K, gid, slot0, KS, s_ids, s_w);
                        if (e1) walk_event(w1, Tt.y, a1, tau_stop, K, gid, slot1, KS, s_ids, s_w);
                    }
                    if (t0 && !e0) w0.T = Tt.x;
                    if (t1 && !e1) w1.T = Tt.y;
                }
                if (w0.done && w1.done) break;
            }
        }
    }
    s_D[slot0] = 1.0f - w0.TQ;
    s_D[slot1] = 1.0f - w1.TQ;
    s_cnt[slot0] = uint8_t(w0.m);
    s_cnt[slot1] = uint8_t(w1.m);
    __syncthreads();
    // coalesced output: each row of the tile is tile_w * K consecutive entries
    // of ids and weights in the image
    const int rowlen = tile_w * K;
    for (int rem = threadIdx.x; rem < rowlen; rem += kThreads) {
        const int cx = rem / K, j = rem - cx * K;
        const int gx = tx * tile_w + cx;
        if (gx >= W) continue;
        for (int row = 0; row < tile_h; ++row) {
            const int gy = ty * tile_h + row;
            if (gy >= H) break;
            const int slot = row * tile_w + cx;
            const int64_t o = (int64_t(gy) * W + gx) * K + j;
            const bool has = j < int(s_cnt[slot]);
            ids[o] = has ? s_ids[slot * KS + j] : -1;
            wout[o] = has ? __fdiv_rn(s_w[slot * KS + j], s_D[slot]) : 0.0f;
        }
    }
    for (int e = threadIdx.x; e < kPix; e += kThreads) {
        const int gx = tx * tile_w + e % tile_w, gy = ty * tile_h + e / tile_w;
        if (gx < W && gy < H) cnt[int64_t(gy) * W + gx] = s_cnt[e];
    }
}

}  // namespace

cudaError_t launch_select(const qr_frame &f, int32_t *ids, float *w, uint8_t *cnt,
                          cudaStream_t s) {
    const int tiles = num_tiles(f);
    if (tiles == 0) return cudaSuccess;
    const int K = f.params.K;
    const size_t dyn = size_t(K | 1) * kPix * 8;
    if (dyn > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(select_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             int(dyn));
        if (e != cudaSuccess) return e;
    }
    cudaError_t e = pdl_launch(
        select_kernel, dim3(tiles), dim3(kThreads), dyn, s, (const float4 *)slot<float4>(f, S_REC_M),
        (const float4 *)slot<float4>(f, S_REC_C), (const float *)slot<float>(f, S_REC_A),
        (const float *)slot<float>(f, S_REC_H), (const uint32_t *)slot<uint32_t>(f, S_IGID),
        (const uint2 *)slot<uint2>(f, S_RANGES), f.camera.width, f.camera.height, f.params.tile_w,
        f.tiles_x, K, f.params.alpha_min, f.params.alpha_max, ids, w, cnt);
    count_launch();
    return e != cudaSuccess ? e : cudaGetLastError();
}

}  // namespace qr
