// K1: EWA projection of every Gaussian (Sec. 3 of the paper).
//
// Per Gaussian: camera-space mean c = R mu + t, 3D covariance
// Sigma = Rq S S^T Rq^T (S = diag(exp(log_scale)), Rq from the quaternion),
// EWA 2D covariance Sigma' = (J W) Sigma (J W)^T + dilation I with J the
// Jacobian of the pinhole map at c, conic A = Sigma'^{-1}, projected mean
// mu' = (fx c_x/c_z + cx, fy c_y/c_z + cy), the conic's scaled principal axes
// (A = 2 (w1 w1^T + w2 w2^T), the form every pixel evaluates), and the screen
// tiles its support
// {u : alpha exp(-q(u)/2) >= alpha_min}, q = (u-mu')^T A (u-mu'), can reach.
//
// GB300 design: one kernel, one CTA per 1024 consecutive ids.  Stage A (a
// thread per Gaussian, four coalesced passes) applies a cheap FP32 bound on
// the footprint and writes the culled records; the survivors (a tenth of an
// indoor scene) are compacted in shared memory and the CTA's threads run
// stage B on them: the exact projection in compensated double-FP32
// arithmetic.  Stage B is what makes the per-pixel alpha' agree with an FP64
// evaluation to ~1e-6 relative: the projected mean is kept as an unevaluated
// pair hi + lo, so the pixel offset u - mu' loses nothing even 1000 px from
// the origin.  Every output is indexed by Gaussian id, the per-256-id kept
// counts and tile sums are exact integer sums over the CTA's own id blocks,
// and the tile rectangles go to a difference array by integer atomics, so
// the result does not depend on the order in which survivors are processed.
#include "qr_internal.cuh"

namespace qr {
namespace {

constexpr int kThreads = kProjectThreads;
constexpr int kProjPer = 4;   // Gaussians per thread in the cull stage: 4 id blocks per CTA

struct CamArgs {
    float R[9], t[3], fx, fy, cx, cy, znear;
    int W, H;
};

__device__ __forceinline__ void write_culled(int64_t g, uint32_t *dkey, uint32_t *tcount,
                                             uint2 *rect) {
    dkey[g] = 0xFFFFFFFFu;
    tcount[g] = 0u;
    rect[g] = make_uint2(0u, 0u);
}

// Stage A: conservative FP32 footprint bound.  True if the Gaussian may reach
// the screen; a non-finite opacity fails (NaN fails the first test).
__device__ __forceinline__ bool cull_pass(int64_t g, const float *__restrict__ mean,
                                          const float *__restrict__ log_scale,
                                          const float *__restrict__ opacity, const CamArgs &cam,
                                          float dilation, float alpha_min) {
    const float mx = mean[3 * g], my = mean[3 * g + 1], mz = mean[3 * g + 2];
    const float alpha = opacity[g];
    const float cz = fmaf(cam.R[6], mx, fmaf(cam.R[7], my, fmaf(cam.R[8], mz, cam.t[2])));
    if (!(alpha >= alpha_min && alpha <= 3.402823466e38f && cz > cam.znear - 1e-3f)) return false;
    const float cx_ = fmaf(cam.R[0], mx, fmaf(cam.R[1], my, fmaf(cam.R[2], mz, cam.t[0])));
    const float cy_ = fmaf(cam.R[3], mx, fmaf(cam.R[4], my, fmaf(cam.R[5], mz, cam.t[1])));
    const float zz = fmaxf(cz, 0.5f * cam.znear);
    const float u = cx_ / zz, v = cy_ / zz;
    const float smax = __expf(fmaxf(log_scale[3 * g], fmaxf(log_scale[3 * g + 1], log_scale[3 * g + 2])));
    const float r2 = 2.0f * __logf(fmaxf(alpha / alpha_min, 1.0f));
    // Sigma'_00 <= smax^2 |J_x|^2 + dilation with |J_x| = fx/z sqrt(1+u^2)
    const float jx = cam.fx / zz, jy = cam.fy / zz;
    const float ex = sqrtf(r2 * (smax * smax * jx * jx * (1.f + u * u) + dilation)) * 1.01f + 2.f;
    const float ey = sqrtf(r2 * (smax * smax * jy * jy * (1.f + v * v) + dilation)) * 1.01f + 2.f;
    const float px = fmaf(cam.fx, u, cam.cx), py = fmaf(cam.fy, v, cam.cy);
    const float tol = 1e-3f * (fabsf(px) + fabsf(py)) + 2.f;
    return (px + ex + tol >= 0.f) && (px - ex - tol <= float(cam.W)) && (py + ey + tol >= 0.f) &&
           (py - ey - tol <= float(cam.H));
}

// Stage B: exact projection of one candidate gi; s_vis / s_ts are the CTA's
// per-256-id counters, blk = gi's block within the CTA.
__device__ __forceinline__ void project_one(int64_t gi, int blk, const float *__restrict__ mean,
                                            const float *__restrict__ log_scale,
                                            const float *__restrict__ quat,
                                            const float *__restrict__ opacity, const CamArgs &cam,
                                            float dilation, float alpha_min, int tile_w, int tile_h,
                                            float4 *__restrict__ rec_m, float4 *__restrict__ rec_w,
                                            float *__restrict__ rec_a, float *__restrict__ rec_h,
                                            uint2 *__restrict__ rect, uint32_t *__restrict__ tcount,
                                            uint32_t *__restrict__ dkey, uint32_t *s_vis,
                                            uint32_t *s_ts, int tiles_x, int *__restrict__ dcopy) {
    const float mx = mean[3 * gi], my = mean[3 * gi + 1], mz = mean[3 * gi + 2];
    const float alpha = opacity[gi];
    // c = R mu + t
    df c[3];
#pragma unroll
    for (int r = 0; r < 3; ++r)
        c[r] = df_add(df_add(df_add(df_two_prod(cam.R[3 * r], mx), df_two_prod(cam.R[3 * r + 1], my)),
                             df_two_prod(cam.R[3 * r + 2], mz)),
                      df_from(cam.t[r]));
    if (!(c[2].hi > cam.znear || (c[2].hi == cam.znear && c[2].lo > 0.f))) {
        write_culled(gi, dkey, tcount, rect);
        return;
    }
    // homogeneous rotation of the (unnormalised) quaternion: Rq = M / |q|^2
    const float qw = quat[4 * gi], qx = quat[4 * gi + 1], qy = quat[4 * gi + 2], qz = quat[4 * gi + 3];
    const df ww = df_two_prod(qw, qw), xx = df_two_prod(qx, qx), yy = df_two_prod(qy, qy),
             zz = df_two_prod(qz, qz);
    const df xy = df_two_prod(qx, qy), xz = df_two_prod(qx, qz), yz = df_two_prod(qy, qz),
             wx = df_two_prod(qw, qx), wy = df_two_prod(qw, qy), wz = df_two_prod(qw, qz);
    df M[9];
    M[0] = df_sub(df_add(ww, xx), df_add(yy, zz));
    M[4] = df_sub(df_add(ww, yy), df_add(xx, zz));
    M[8] = df_sub(df_add(ww, zz), df_add(xx, yy));
    M[1] = df_mul_f(df_sub(xy, wz), 2.f);
    M[2] = df_mul_f(df_add(xz, wy), 2.f);
    M[3] = df_mul_f(df_add(xy, wz), 2.f);
    M[5] = df_mul_f(df_sub(yz, wx), 2.f);
    M[6] = df_mul_f(df_sub(xz, wy), 2.f);
    M[7] = df_mul_f(df_add(yz, wx), 2.f);
    const df qn = df_add(df_add(ww, xx), df_add(yy, zz));
    // J W: rows (fx/z)(W0 - u W2), (fy/z)(W1 - v W2) with u = x/z, v = y/z
    const df iz = df_div(df_from(1.f), c[2]);
    const df u = df_mul(c[0], iz), v = df_mul(c[1], iz);
    const df jx = df_mul_f(iz, cam.fx), jy = df_mul_f(iz, cam.fy);
    df T0[3], T1[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        T0[k] = df_mul(jx, df_sub(df_from(cam.R[k]), df_mul_f(u, cam.R[6 + k])));
        T1[k] = df_mul(jy, df_sub(df_from(cam.R[3 + k]), df_mul_f(v, cam.R[6 + k])));
    }
    // P = (J W) M ; Sigma' = P diag(s^2) P^T / |q|^4
    df P0[3], P1[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        P0[k] = df_dot3(T0[0], M[k], T0[1], M[3 + k], T0[2], M[6 + k]);
        P1[k] = df_dot3(T1[0], M[k], T1[1], M[3 + k], T1[2], M[6 + k]);
    }
    df s00 = df_from(0.f), s01 = df_from(0.f), s11 = df_from(0.f);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const float sk = expf(log_scale[3 * gi + k]);
        const df sk2 = df_two_prod(sk, sk);
        const df a0 = df_mul(P0[k], sk2);
        s00 = df_add(s00, df_mul(a0, P0[k]));
        s01 = df_add(s01, df_mul(a0, P1[k]));
        s11 = df_add(s11, df_mul(df_mul(P1[k], sk2), P1[k]));
    }
    const df inq2 = df_div(df_from(1.f), df_mul(qn, qn));
    s00 = df_add_f(df_mul(s00, inq2), dilation);
    s01 = df_mul(s01, inq2);
    s11 = df_add_f(df_mul(s11, inq2), dilation);
    const df det = df_sub(df_mul(s00, s11), df_mul(s01, s01));
    if (!(det.hi > 0.f)) {
        write_culled(gi, dkey, tcount, rect);
        return;
    }
    // principal axes of Sigma': lambda1 >= lambda2 > 0, unit eigenvector e1;
    // the conic's scaled axes are w_k = e_k / sqrt(2 lambda_k)
    const df hd = df_mul_f(df_sub(s00, s11), 0.5f);
    const df rad = df_sqrt(df_add(df_mul(hd, hd), df_mul(s01, s01)));
    const df l1 = df_add(df_mul_f(df_add(s00, s11), 0.5f), rad);
    const df l2 = df_div(det, l1);
    const df ax = df_sub(l1, s11), bx = df_sub(l1, s00);
    df vx, vy;
    if (df_abs_hi(ax) + df_abs_hi(s01) >= df_abs_hi(s01) + df_abs_hi(bx)) {
        vx = ax; vy = s01;
    } else {
        vx = s01; vy = bx;
    }
    df nv = df_sqrt(df_add(df_mul(vx, vx), df_mul(vy, vy)));
    if (!(nv.hi > 0.f)) { vx = df_from(1.f); vy = df_from(0.f); nv = df_from(1.f); }
    const df e1x = df_div(vx, nv), e1y = df_div(vy, nv);
    const df r1 = df_div(df_from(1.f), df_sqrt(df_mul_f(l1, 2.f)));
    const df r2 = df_div(df_from(1.f), df_sqrt(df_mul_f(l2, 2.f)));
    const float4 waxes = make_float4(df_mul(e1x, r1).hi, df_mul(e1y, r1).hi,
                                     -df_mul(e1y, r2).hi, df_mul(e1x, r2).hi);
    const df mxp = df_add_f(df_mul_f(u, cam.fx), cam.cx);
    const df myp = df_add_f(df_mul_f(v, cam.fy), cam.cy);

    // footprint: q <= r^2 = 2 ln(alpha/alpha_min); extent r sqrt(Sigma'_ii); 1 px pad
    const float r = sqrtf(2.0f * logf(fmaxf(alpha / alpha_min, 1.0f))) * 1.0001f;
    float ex = r * sqrtf(s00.hi), ey = r * sqrtf(s11.hi);
    if (!(isfinite(mxp.hi) && isfinite(myp.hi) && ex >= 0.f && ey >= 0.f)) {
        write_culled(gi, dkey, tcount, rect);
        return;
    }
    ex = fminf(ex, 1e7f);
    ey = fminf(ey, 1e7f);
    const float x0f = floorf(mxp.hi - ex - 1.5f), x1f = floorf(mxp.hi + ex + 0.5f);
    const float y0f = floorf(myp.hi - ey - 1.5f), y1f = floorf(myp.hi + ey + 0.5f);
    const int x0 = int(fmaxf(x0f, 0.f)), x1 = int(fminf(x1f, float(cam.W - 1)));
    const int y0 = int(fmaxf(y0f, 0.f)), y1 = int(fminf(y1f, float(cam.H - 1)));
    if (x1f < 0.f || y1f < 0.f || x0f > float(cam.W - 1) || y0f > float(cam.H - 1) ||
        x0 > x1 || y0 > y1) {
        write_culled(gi, dkey, tcount, rect);
        return;
    }
    const int tx0 = x0 / tile_w, tx1 = x1 / tile_w, ty0 = y0 / tile_h, ty1 = y1 / tile_h;
    rec_m[gi] = make_float4(mxp.hi, myp.hi, mxp.lo, myp.lo);
    rec_w[gi] = waxes;
    rec_a[gi] = alpha;
    rec_h[gi] = reject_half_q(alpha, alpha_min);
    rect[gi] = make_uint2(uint32_t(tx0) | (uint32_t(ty0) << 16), uint32_t(tx1) | (uint32_t(ty1) << 16));
    const uint32_t nt = uint32_t((tx1 - tx0 + 1) * (ty1 - ty0 + 1));
    tcount[gi] = nt;
    dkey[gi] = __float_as_uint(c[2].hi);
    // per-256-id counts of kept Gaussians and of their tiles (scanned by the
    // binning; summed in shared memory, the CTA owns its id blocks), and the
    // footprint rectangle in the difference array of
    // per-tile counts: +1 at (x0,y0) and (x1+1,y1+1), -1 at (x1+1,y0) and (x0,y1+1)
    atomicAdd(&s_vis[blk], 1u);
    atomicAdd(&s_ts[blk], nt);
    const int stride = tiles_x + 1;
    atomicAdd(&dcopy[ty0 * stride + tx0], 1);
    atomicAdd(&dcopy[ty0 * stride + tx1 + 1], -1);
    atomicAdd(&dcopy[(ty1 + 1) * stride + tx0], -1);
    atomicAdd(&dcopy[(ty1 + 1) * stride + tx1 + 1], 1);
}

// One CTA per kProjPer x 256 consecutive ids (kProjPer id blocks of 256):
// stage A culls them (coalesced, kProjPer passes) and writes the culled
// records; the survivors are compacted in shared memory (one shared atomic
// per warp) and the CTA's threads run stage B on them.  The per-256-id
// counts are summed in shared memory and written (not accumulated) for the
// CTA's own id blocks, so only the difference array needs clearing (a memset
// before the launch).
__global__ void __launch_bounds__(kThreads)
project_kernel(int64_t n, const float *__restrict__ mean, const float *__restrict__ log_scale,
               const float *__restrict__ quat, const float *__restrict__ opacity, CamArgs cam,
               float dilation, float alpha_min, int tile_w, int tile_h,
               float4 *__restrict__ rec_m, float4 *__restrict__ rec_w, float *__restrict__ rec_a,
               float *__restrict__ rec_h, uint2 *__restrict__ rect, uint32_t *__restrict__ tcount,
               uint32_t *__restrict__ dkey, uint32_t *__restrict__ vis_count,
               uint32_t *__restrict__ tile_sum, int tiles_x, int tiles_y, int *__restrict__ diff,
               uint32_t *__restrict__ counters) {
    pdl_wait();   // the predecessor's outputs are complete and visible
    __shared__ uint32_t s_cand[kThreads * kProjPer];
    __shared__ uint32_t s_n;
    __shared__ uint32_t s_vis[kProjPer], s_ts[kProjPer];
    if (threadIdx.x < kProjPer) {
        s_vis[threadIdx.x] = 0u;
        s_ts[threadIdx.x] = 0u;
    }
    if (threadIdx.x == 0) s_n = 0u;
    if (blockIdx.x == 0 && threadIdx.x == 0) counters[CNT_N] = uint32_t(n);
    __syncthreads();
    const int64_t g0 = int64_t(blockIdx.x) * (kThreads * kProjPer);
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int k = 0; k < kProjPer; ++k) {
        const int64_t g = g0 + k * kThreads + threadIdx.x;
        bool pass = false;
        if (g < n) {
            pass = cull_pass(g, mean, log_scale, opacity, cam, dilation, alpha_min);
            if (!pass) write_culled(g, dkey, tcount, rect);
        }
        const unsigned ballot = __ballot_sync(0xffffffffu, pass);
        uint32_t base = 0;
        if (lane == 0 && ballot) base = atomicAdd(&s_n, uint32_t(__popc(ballot)));
        base = __shfl_sync(0xffffffffu, base, 0);
        if (pass) s_cand[base + uint32_t(__popc(ballot & ((1u << lane) - 1u)))] = uint32_t(g - g0);
    }
    __syncthreads();
    const uint32_t nc = s_n;
    int *dcopy = diff + size_t(blockIdx.x % kDiffCopies) * size_t(tiles_x + 1) * size_t(tiles_y + 1);
    for (uint32_t i = threadIdx.x; i < nc; i += kThreads) {
        const uint32_t loc = s_cand[i];
        project_one(g0 + loc, int(loc >> 8), mean, log_scale, quat, opacity, cam, dilation,
                    alpha_min, tile_w, tile_h, rec_m, rec_w, rec_a, rec_h, rect, tcount, dkey,
                    s_vis, s_ts, tiles_x, dcopy);
    }
    __syncthreads();
    if (threadIdx.x < kProjPer) {
        const int64_t blk = g0 / kThreads + threadIdx.x;
        if (blk * kThreads < n) {
            vis_count[blk] = s_vis[threadIdx.x];
            tile_sum[blk] = s_ts[threadIdx.x];
        }
    }
}

}  // namespace

cudaError_t launch_project(const qr_frame &f, const float *mean, const float *log_scale,
                           const float *quat, const float *opacity, cudaStream_t s) {
    const int64_t n = f.n;
    uint32_t *counters = slot<uint32_t>(f, S_COUNTERS);
    // the counters and the difference array are adjacent slots: one memset
    const size_t ndiff = size_t(f.tiles_x + 1) * size_t(f.tiles_y + 1) * kDiffCopies;
    const size_t clear = f.off[S_DIFF] - f.off[S_COUNTERS] + ndiff * sizeof(int);
    cudaError_t e = cudaMemsetAsync(counters, 0, clear, s);
    if (e != cudaSuccess) return e;
    if (n == 0) return cudaSuccess;
    CamArgs cam;
    for (int i = 0; i < 9; ++i) cam.R[i] = f.camera.R[i];
    for (int i = 0; i < 3; ++i) cam.t[i] = f.camera.t[i];
    cam.fx = f.camera.fx; cam.fy = f.camera.fy; cam.cx = f.camera.cx; cam.cy = f.camera.cy;
    cam.znear = f.camera.near_plane; cam.W = f.camera.width; cam.H = f.camera.height;
    const unsigned blocks = unsigned((n + kThreads * kProjPer - 1) / (kThreads * kProjPer));
    e = pdl_launch(project_kernel, dim3(blocks), dim3(kThreads), 0, s, n, mean, log_scale, quat,
                   opacity, cam, f.params.dilation, f.params.alpha_min, f.params.tile_w,
                   f.params.tile_h, slot<float4>(f, S_REC_M), slot<float4>(f, S_REC_C),
                   slot<float>(f, S_REC_A), slot<float>(f, S_REC_H), slot<uint2>(f, S_RECT),
                   slot<uint32_t>(f, S_TCOUNT), slot<uint32_t>(f, S_GKEY),
                   slot<uint32_t>(f, S_VISCNT), slot<uint32_t>(f, S_BSUM), f.tiles_x, f.tiles_y,
                   slot<int>(f, S_DIFF), counters);
    count_launch(1);
    return e != cudaSuccess ? e : cudaGetLastError();
}

}  // namespace qr
