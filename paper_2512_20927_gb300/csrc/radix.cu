// Stable LSD radix sort of (u32 key, u32 value) pairs, hand-written
// reduce-then-scan: per-block digit histograms, a warp-per-digit scan of the
// [digit][block] table, then a stable scatter whose per-warp ranks come from
// __match_any_sync.  No CTA ever waits for another.  Item counts are read from
// device memory, so a sort can be captured in a CUDA graph with worst-case
// grids.  Used to reduce per-pixel contributions by Gaussian in the backward.
#include "qr_internal.cuh"

namespace qr {
namespace {

constexpr int T = kSortThreads;      // 256
constexpr int IPT = kSortItems;      // 8
constexpr int TILE = kSortTile;      // 2048
constexpr int WARPS = T / 32;

__device__ __forceinline__ void block_tiles(uint32_t n, int b, int nb, uint32_t &t0, uint32_t &t1) {
    const uint32_t tiles = (n + TILE - 1) / TILE;
    const uint32_t per = (tiles + nb - 1) / nb;
    t0 = min(tiles, uint32_t(b) * per);
    t1 = min(tiles, t0 + per);
}

__device__ __forceinline__ unsigned lanemask_lt() {
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// ------------------------------------------------------------------ radix pass
__global__ void __launch_bounds__(T)
radix_upsweep(const uint32_t *__restrict__ keys, const uint32_t *__restrict__ d_count, int shift,
              int bits, uint32_t *__restrict__ hist) {
    __shared__ uint32_t s_h[WARPS][1 << kRadixBitsMax];
    const int radix = 1 << bits;
    const uint32_t mask = uint32_t(radix - 1);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int i = threadIdx.x; i < WARPS * radix; i += T) (&s_h[0][0])[(i / radix) * (1 << kRadixBitsMax) + i % radix] = 0;
    __syncthreads();
    const uint32_t n = *d_count;
    uint32_t t0, t1;
    block_tiles(n, blockIdx.x, gridDim.x, t0, t1);
    const uint32_t end = min(n, t1 * TILE);
    for (uint32_t base = t0 * TILE; base < end; base += T) {   // uniform trip count
        const uint32_t i = base + threadIdx.x;
        const bool valid = i < end;
        const uint32_t d = valid ? (keys[i] >> shift) & mask : 0xFFFFFFFFu;
        const unsigned peers = __match_any_sync(0xffffffffu, d);
        if (valid && lane == __ffs(peers) - 1) atomicAdd(&s_h[warp][d], uint32_t(__popc(peers)));
    }
    __syncthreads();
    for (int d = threadIdx.x; d < radix; d += T) {
        uint32_t s = 0;
#pragma unroll
        for (int w = 0; w < WARPS; ++w) s += s_h[w][d];
        hist[d * gridDim.x + blockIdx.x] = s;
    }
}

// One warp per digit: exclusive scan of the digit's per-block counts (row d of
// the [digit][block] table) in place; the row total goes to digitsum[d].
__global__ void __launch_bounds__(256)
radix_scan_rows(uint32_t *__restrict__ hist, int radix, int blocks, uint32_t *__restrict__ digitsum) {
    const int d = blockIdx.x * 8 + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (d >= radix) return;
    uint32_t *row = hist + size_t(d) * blocks;
    uint32_t carry = 0;
    for (int base = 0; base < blocks; base += 32) {
        const int i = base + lane;
        const uint32_t v = i < blocks ? row[i] : 0u;
        uint32_t x = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (i < blocks) row[i] = carry + x - v;
        carry += __shfl_sync(0xffffffffu, x, 31);
    }
    if (lane == 0) digitsum[d] = carry;
}

__global__ void __launch_bounds__(T)
radix_downsweep(const uint32_t *__restrict__ keys_in, const uint32_t *__restrict__ vals_in,
                uint32_t *__restrict__ keys_out, uint32_t *__restrict__ vals_out,
                const uint32_t *__restrict__ d_count, int shift, int bits,
                const uint32_t *__restrict__ hist, const uint32_t *__restrict__ digitsum) {
    __shared__ uint32_t s_base[1 << kRadixBitsMax];
    __shared__ uint32_t s_scan[32];
    __shared__ uint32_t s_tot[1 << kRadixBitsMax];
    __shared__ uint32_t s_w[WARPS][1 << kRadixBitsMax];
    const int radix = 1 << bits;
    const uint32_t mask = uint32_t(radix - 1);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const unsigned lt = lanemask_lt();
    {   // base of digit d for this block = sum of smaller digits + this digit's earlier blocks
        const uint32_t ds = threadIdx.x < radix ? digitsum[threadIdx.x] : 0u;
        uint32_t tot;
        const uint32_t inc = block_inclusive_scan(ds, s_scan, tot);
        if (threadIdx.x < radix) s_base[threadIdx.x] = inc - ds + hist[threadIdx.x * gridDim.x + blockIdx.x];
    }
    const uint32_t n = *d_count;
    uint32_t t0, t1;
    block_tiles(n, blockIdx.x, gridDim.x, t0, t1);
    for (uint32_t tile = t0; tile < t1; ++tile) {
        for (int i = threadIdx.x; i < WARPS * radix; i += T) s_w[i / radix][i % radix] = 0;
        __syncthreads();
        uint32_t key[IPT], val[IPT], rank[IPT], dig[IPT];
        const uint32_t wbase = tile * TILE + warp * (32 * IPT);
#pragma unroll
        for (int r = 0; r < IPT; ++r) {
            const uint32_t idx = wbase + r * 32 + lane;
            const bool valid = idx < n;
            key[r] = valid ? keys_in[idx] : 0u;
            val[r] = valid ? vals_in[idx] : 0u;
            dig[r] = valid ? (key[r] >> shift) & mask : 0xFFFFFFFFu;
            const unsigned peers = __match_any_sync(0xffffffffu, dig[r]);
            const uint32_t before = valid ? s_w[warp][dig[r]] : 0u;
            rank[r] = before + __popc(peers & lt);
            __syncwarp();
            if (valid && lane == __ffs(peers) - 1) s_w[warp][dig[r]] = before + __popc(peers);
            __syncwarp();
        }
        __syncthreads();
        for (int d = threadIdx.x; d < radix; d += T) {
            uint32_t run = 0;
#pragma unroll
            for (int w = 0; w < WARPS; ++w) {
                const uint32_t c = s_w[w][d];
                s_w[w][d] = run;
                run += c;
            }
            s_tot[d] = run;
        }
        __syncthreads();
#pragma unroll
        for (int r = 0; r < IPT; ++r) {
            if (dig[r] != 0xFFFFFFFFu) {
                const uint32_t pos = s_base[dig[r]] + s_w[warp][dig[r]] + rank[r];
                keys_out[pos] = key[r];
                vals_out[pos] = val[r];
            }
        }
        __syncthreads();
        for (int d = threadIdx.x; d < radix; d += T) s_base[d] += s_tot[d];
        __syncthreads();
    }
}

}  // namespace

int sort_blocks_for(int64_t capacity) {
    const int64_t tiles = (capacity + TILE - 1) / TILE;
    return int(tiles < 1 ? 1 : (tiles > kSortMaxBlocks ? kSortMaxBlocks : tiles));
}

cudaError_t radix_sort_pairs(uint32_t *keys_a, uint32_t *vals_a, uint32_t *keys_b,
                             uint32_t *vals_b, const uint32_t *d_count, int64_t capacity,
                             int bit_lo, int bit_hi, uint32_t *hist, uint32_t *digitsum,
                             int blocks, int *result_in_b, cudaStream_t s) {
    (void)capacity;
    int in_b = 0;
    for (int lo = bit_lo; lo < bit_hi;) {
        const int remaining = bit_hi - lo;
        const int passes_left = (remaining + kRadixBitsMax - 1) / kRadixBitsMax;
        const int bits = (remaining + passes_left - 1) / passes_left;
        uint32_t *ki = in_b ? keys_b : keys_a, *vi = in_b ? vals_b : vals_a;
        uint32_t *ko = in_b ? keys_a : keys_b, *vo = in_b ? vals_a : vals_b;
        radix_upsweep<<<blocks, T, 0, s>>>(ki, d_count, lo, bits, hist);
        radix_scan_rows<<<((1 << bits) + 7) / 8, 256, 0, s>>>(hist, 1 << bits, blocks, digitsum);
        radix_downsweep<<<blocks, T, 0, s>>>(ki, vi, ko, vo, d_count, lo, bits, hist, digitsum);
        count_launch(3);
        in_b ^= 1;
        lo += bits;
    }
    if (result_in_b) *result_in_b = in_b;
    return cudaGetLastError();
}

}  // namespace qr
