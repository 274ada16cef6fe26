// The selection half of Algorithm 1 for one screen tile, shared by the
// single-view selection kernel (select.cu) and the many-view persistent
// kernel (batch.cu), so both keep exactly the same Gaussians with the same
// FP32 weights.
//
// Per pixel, front to back over the tile's depth-ordered list:
//   alpha' = min(alpha_max, alpha exp(-q/2)); entries with alpha' < alpha_min
//   are not members of I and leave T unchanged;
//   T_test = T (1 - alpha');
//   if T_test < tau_k (tau_k = (K-k)/(K+1), the boundary 1-(k+1)/(K+1)):
//       keep the Gaussian with weight w = T^Q alpha', T^Q *= 1 - alpha',
//       advance k past every boundary T_test is below;
//   stop once T_test < 1/(K+1); otherwise T = T_test.
//
// 128 threads walk the tile's 256 pixels, two vertically adjacent pixels of
// the same column each.  The tile's list is staged through shared memory 128
// entries at a time (gid, projected mean hi/lo, conic axes, opacity, reject
// bound: 44 B each) with coalesced loads; the ids of the next batch are
// fetched while the current one is walked.
//   * Each warp first culls the staged entries against its box of pixel
//     centres, one entry per lane: the minimum of q/2 over the box against
//     the entry's reject bound.  Most entries a pixel would walk are out of
//     reach of the whole box.
//   * The warp walks the survivors four per step (independent chains).  The
//     two pixels of a thread share the x offset; their y offsets, axis
//     projections and q/2 use packed FP32x2 instructions (each half rounds
//     exactly like the scalar instruction).  Entries within reach take the
//     Algorithm 1 step for both pixels at once; only keeping a Gaussian or
//     stopping branches off.
// The 128 threads stop loading as soon as all of their pixels have stopped.
// Kept (id, unnormalised weight) pairs go to per-pixel shared-memory slots
// [256][K|1]; s_D gets 1 - T^Q and s_cnt the kept count of each pixel.
//
// The barrier policy Bar joins the 128 walking threads: the whole CTA in the
// selection kernel, a named barrier in the many-view kernel (whose other
// warps blend meanwhile).
#pragma once

#include "qr_internal.cuh"

namespace qr {

constexpr int kSelPix = 256;       // pixels per tile
constexpr int kSelThreads = 128;   // two pixels per thread
constexpr int kSelBatch = 128;     // list entries staged per batch

struct SelStage {
    float4 m[kSelBatch];
    float4 c[kSelBatch];
    float a[kSelBatch];
    float h[kSelBatch];
    uint32_t g[kSelBatch];
};

struct CtaBarrier {
    __device__ static void sync() { __syncthreads(); }
    __device__ static int count(bool p) { return __syncthreads_count(p); }
};

template <int ID, int N>
struct NamedBarrier {
    __device__ static void sync() { asm volatile("bar.sync %0, %1;" ::"n"(ID), "n"(N) : "memory"); }
    __device__ static int count(bool p) {
        int r;
        asm volatile("{\n .reg .pred q;\n setp.ne.u32 q, %1, 0;\n bar.red.popc.u32 %0, %2, %3, q;\n}\n"
                     : "=r"(r) : "r"(int(p)), "n"(ID), "n"(N) : "memory");
        return r;
    }
};

__device__ __forceinline__ float2 sel_add2(float2 a, float2 b) {
    float2 d;
    asm("{\n .reg .b64 x, y;\n mov.b64 x, {%2, %3};\n mov.b64 y, {%4, %5};\n"
        " add.rn.f32x2 x, x, y;\n mov.b64 {%0, %1}, x;\n}\n"
        : "=f"(d.x), "=f"(d.y) : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return d;
}
__device__ __forceinline__ float2 sel_mul2(float2 a, float2 b) {
    float2 d;
    asm("{\n .reg .b64 x, y;\n mov.b64 x, {%2, %3};\n mov.b64 y, {%4, %5};\n"
        " mul.rn.f32x2 x, x, y;\n mov.b64 {%0, %1}, x;\n}\n"
        : "=f"(d.x), "=f"(d.y) : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return d;
}
__device__ __forceinline__ float2 sel_fma2(float2 a, float2 b, float2 c) {
    float2 d;
    asm("{\n .reg .b64 x, y, z;\n mov.b64 x, {%2, %3};\n mov.b64 y, {%4, %5};\n"
        " mov.b64 z, {%6, %7};\n fma.rn.f32x2 x, x, y, z;\n mov.b64 {%0, %1}, x;\n}\n"
        : "=f"(d.x), "=f"(d.y)
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y), "f"(c.x), "f"(c.y));
    return d;
}

// Walks tile (tx, ty) whose depth-ordered ids are isect_gid[range.x, range.y).
// Called by threads 0..127 (all of them); ends with the per-pixel results in
// s_ids / s_w / s_D / s_cnt, written by their owners (the caller joins the
// threads with Bar::sync() before reading other pixels' slots).  With
// kCount the weights are boundary-crossing counts and s_D the number of
// boundaries crossed in all (App. C's Riemann weights); the selection is the
// same.
template <class Bar, bool kCount = false>
__device__ __forceinline__ void select_tile(const float4 *__restrict__ rec_m,
                                            const float4 *__restrict__ rec_w,
                                            const float *__restrict__ rec_a,
                                            const float *__restrict__ rec_h,
                                            const uint32_t *__restrict__ isect_gid, uint2 range,
                                            int W, int H, int tile_w, int tx, int ty, int K,
                                            float alpha_min, float alpha_max, SelStage &st,
                                            int32_t *s_ids, float *s_w, float *s_D, uint8_t *s_cnt) {
    const int KS = K | 1;   // odd stride: the per-pixel slots fall in distinct banks
    const int tile_h = kSelPix / tile_w;
    const int lx = threadIdx.x % tile_w, ly = 2 * (threadIdx.x / tile_w);
    const int px = tx * tile_w + lx, py = ty * tile_h + ly;
    const int slot0 = ly * tile_w + lx, slot1 = slot0 + tile_w;
    const bool in0 = px < W && py < H, in1 = px < W && py + 1 < H;
    const float ux = float(px) + 0.5f;
    const float2 uy = make_float2(float(py) + 0.5f, float(py + 1) + 0.5f);

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
    for (uint32_t b = range.x; b < range.y; b += kSelBatch) {
        if (Bar::count(w0.done && w1.done) == kSelThreads) break;
        if (b + threadIdx.x < range.y) {
            st.g[threadIdx.x] = gnext;
            st.m[threadIdx.x] = rec_m[gnext];
            st.c[threadIdx.x] = rec_w[gnext];
            st.a[threadIdx.x] = rec_a[gnext];
            st.h[threadIdx.x] = rec_h[gnext];
        }
        Bar::sync();
        {
            const uint32_t idx = b + kSelBatch + threadIdx.x;
            gnext = idx < range.y ? isect_gid[idx] : 0u;
        }
        const int nb = int(min(uint32_t(kSelBatch), range.y - b));
        for (int c0 = 0; c0 < nb; c0 += 32) {
            if (__all_sync(FULL, w0.done && w1.done)) break;
            // cull 32 staged entries against the warp's box (one per lane): an
            // entry whose q/2 stays above its reject bound over the whole box
            // is skipped by every pixel of the warp anyway
            const int jl = c0 + lane;
            bool pass = false;
            if (jl < nb)
                pass = !(box_min_half_q(st.m[jl], st.c[jl], bx0, bx1, by0, by1) * 0.999f > st.h[jl] + 1e-3f);
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
                    const float4 mm = st.m[j];
                    const float4 cc = st.c[j];
                    h[u] = st.h[j];
                    // eval_half_q for both pixels: dx shared, the rest packed
                    const float dx = (ux - mm.x) - mm.z;
                    const float2 dy = sel_add2(sel_add2(uy, make_float2(-mm.y, -mm.y)),
                                               make_float2(-mm.w, -mm.w));
                    const float2 dx2 = make_float2(dx, dx);
                    const float2 p1 = sel_fma2(dx2, make_float2(cc.x, cc.x), sel_mul2(dy, make_float2(cc.y, cc.y)));
                    const float2 p2 = sel_fma2(dx2, make_float2(cc.z, cc.z), sel_mul2(dy, make_float2(cc.w, cc.w)));
                    hq[u] = sel_fma2(p1, p1, sel_mul2(p2, p2));
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
                    const float alpha = st.a[jj[u]];
                    const float a0 = eval_alpha(alpha, hq[u].x, alpha_max);
                    const float a1 = eval_alpha(alpha, hq[u].y, alpha_max);
                    const bool t0 = r0 && !(a0 < alpha_min), t1 = r1 && !(a1 < alpha_min);
                    const float2 Tt = sel_mul2(make_float2(w0.T, w1.T),
                                               sel_add2(make_float2(1.0f, 1.0f),
                                                        make_float2(t0 ? -a0 : -0.0f, t1 ? -a1 : -0.0f)));
                    const bool e0 = t0 && (Tt.x < w0.thr || Tt.x < tau_stop);
                    const bool e1 = t1 && (Tt.y < w1.thr || Tt.y < tau_stop);
                    if (e0 || e1) {
                        const uint32_t gid = st.g[jj[u]];
                        if (e0) walk_event<kCount>(w0, Tt.x, a0, tau_stop, K, gid, slot0, KS, s_ids, s_w);
                        if (e1) walk_event<kCount>(w1, Tt.y, a1, tau_stop, K, gid, slot1, KS, s_ids, s_w);
                    }
                    if (t0 && !e0) w0.T = Tt.x;
                    if (t1 && !e1) w1.T = Tt.y;
                }
                if (w0.done && w1.done) break;
            }
        }
    }
    s_D[slot0] = kCount ? float(w0.k) : 1.0f - w0.TQ;
    s_D[slot1] = kCount ? float(w1.k) : 1.0f - w1.TQ;
    s_cnt[slot0] = uint8_t(w0.m);
    s_cnt[slot1] = uint8_t(w1.m);
}

}  // namespace qr
