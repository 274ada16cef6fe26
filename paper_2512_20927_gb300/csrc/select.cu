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
// 1 - T^Q (the normalisation step folded into the weights).  The same kernel
// serves App. C's Riemann-weight form (QR_RULE_RIEMANN): the same selection,
// each kept Gaussian weighted by the number of boundaries T_test crosses at
// it, divided by the number crossed in all.
//
// GB300 design: one CTA of 128 threads per screen tile; the walk itself
// (select_tile.cuh) stages the tile's list through shared memory, culls it
// per warp against the warp's box of pixel centres and walks two pixels per
// thread with packed FP32x2 arithmetic.  Kept (id, weight) pairs are written
// out once per tile row as contiguous runs of tile_w * K ids and weights, so
// the stores are fully coalesced.
#include "select_tile.cuh"

namespace qr {
namespace {

// kCount: App. C's Riemann weights in place of Algorithm 1's (select_tile).
template <bool kCount>
__global__ void __launch_bounds__(kSelThreads, 8)
select_kernel(const float4 *__restrict__ rec_m, const float4 *__restrict__ rec_w,
              const float *__restrict__ rec_a, const float *__restrict__ rec_h,
              const uint32_t *__restrict__ isect_gid, const uint2 *__restrict__ ranges, int W,
              int H, int tile_w, int tiles_x, int K, float alpha_min, float alpha_max,
              int32_t *__restrict__ ids, float *__restrict__ wout, uint8_t *__restrict__ cnt) {
    pdl_wait();   // the predecessor's outputs are complete and visible
    __shared__ SelStage st;
    __shared__ float s_D[kSelPix];       // 1 - T^Q per pixel
    __shared__ uint8_t s_cnt[kSelPix];
    extern __shared__ unsigned char s_dyn[];
    const int KS = K | 1;
    int32_t *s_ids = reinterpret_cast<int32_t *>(s_dyn);          // [256][KS]
    float *s_w = reinterpret_cast<float *>(s_dyn) + KS * kSelPix;  // [256][KS]
    const int tile = blockIdx.x;
    const int tx = tile % tiles_x, ty = tile / tiles_x;
    const int tile_h = kSelPix / tile_w;
    select_tile<CtaBarrier, kCount>(rec_m, rec_w, rec_a, rec_h, isect_gid, ranges[tile], W, H, tile_w, tx,
                            ty, K, alpha_min, alpha_max, st, s_ids, s_w, s_D, s_cnt);
    __syncthreads();
    // coalesced output: each row of the tile is tile_w * K consecutive entries
    // of ids and weights in the image
    const int rowlen = tile_w * K;
    for (int rem = threadIdx.x; rem < rowlen; rem += kSelThreads) {
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
    for (int e = threadIdx.x; e < kSelPix; e += kSelThreads) {
        const int gx = tx * tile_w + e % tile_w, gy = ty * tile_h + e / tile_w;
        if (gx < W && gy < H) cnt[int64_t(gy) * W + gx] = s_cnt[e];
    }
}

}  // namespace

cudaError_t launch_select(const qr_frame &f, int32_t *ids, float *w, uint8_t *cnt, bool riemann,
                          cudaStream_t s) {
    const int tiles = num_tiles(f);
    if (tiles == 0) return cudaSuccess;
    const int K = f.params.K;
    const size_t dyn = size_t(K | 1) * kSelPix * 8;
    auto go = [&](auto kern) -> cudaError_t {
        if (dyn > 48 * 1024) {
            const cudaError_t e =
                cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(dyn));
            if (e != cudaSuccess) return e;
        }
        return pdl_launch(kern, dim3(tiles), dim3(kSelThreads), dyn, s,
                          (const float4 *)slot<float4>(f, S_REC_M),
                          (const float4 *)slot<float4>(f, S_REC_C),
                          (const float *)slot<float>(f, S_REC_A),
                          (const float *)slot<float>(f, S_REC_H),
                          (const uint32_t *)slot<uint32_t>(f, S_IGID),
                          (const uint2 *)slot<uint2>(f, S_RANGES), f.camera.width,
                          f.camera.height, f.params.tile_w, f.tiles_x, K, f.params.alpha_min,
                          f.params.alpha_max, ids, w, cnt);
    };
    const cudaError_t e = riemann ? go(select_kernel<true>) : go(select_kernel<false>);
    count_launch();
    return e != cudaSuccess ? e : cudaGetLastError();
}

}  // namespace qr
