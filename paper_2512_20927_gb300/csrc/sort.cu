// K2-K4: binning, radix sort and tile ranges (Sec. 3 "tiling strategy"; the
// depth-ordered index list I of Sec. 4.2).
//
// Order produced: intersections sorted by (tile id, depth, Gaussian id), the
// order of a stable sort of 64-bit (tile << 32 | depth-bits) keys over
// id-ordered input.  It is built as
//   1. a stable LSD radix sort of the N 32-bit depth keys (ids as values),
//   2. an exclusive scan of the per-Gaussian tile counts in that order and an
//      emit of one (tile, id) pair per touched tile, in depth order,
//   3. a stable LSD radix sort of the X intersections by tile id only
//      (ceil(log2 tiles) bits, <= 8 bits per pass).
// The depth digits are therefore sorted once per Gaussian instead of once per
// intersection -- the lower-digit passes of the 64-bit LSD sort hoisted in
// front of the duplication, which preserves relative order.
//
// Every pass is reduce-then-scan: per-block digit histograms, one scan of the
// [digit][block] table, then a stable scatter.  No CTA ever waits for another,
// so nothing here can spin.  Item counts are read from device memory, so the
// whole stage can be captured in a CUDA graph with worst-case grids.
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
__device__ void cta_exclusive_scan(uint32_t *data, int total, uint32_t *sum_out) {
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

// ------------------------------------------------------------------ compaction
// The kept Gaussians (finite depth key) are packed in id order, so the depth
// sort works on the visible set only and equal depths keep id order.
__global__ void __launch_bounds__(1024)
compact_scan(uint32_t *vis_count, int nblk, uint32_t *counters) {
    __shared__ uint32_t s_total;
    cta_exclusive_scan(vis_count, nblk, &s_total);
    __syncthreads();
    if (threadIdx.x == 0) counters[CNT_VISIBLE] = s_total;
}

__global__ void __launch_bounds__(kProjectThreads)
compact_scatter(const uint32_t *__restrict__ gkey, const uint32_t *__restrict__ vis_off, int64_t n,
                uint32_t *__restrict__ dkey, uint32_t *__restrict__ dval) {
    __shared__ uint32_t s_w[kProjectThreads / 32];
    const int64_t g = int64_t(blockIdx.x) * kProjectThreads + threadIdx.x;
    const uint32_t key = g < n ? gkey[g] : 0xFFFFFFFFu;
    const bool keep = key != 0xFFFFFFFFu;
    const unsigned ballot = __ballot_sync(0xffffffffu, keep);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) s_w[warp] = __popc(ballot);
    __syncthreads();
    uint32_t off = vis_off[blockIdx.x] + __popc(ballot & ((1u << lane) - 1u));
    for (int w = 0; w < warp; ++w) off += s_w[w];
    if (keep) {
        dkey[off] = key;
        dval[off] = uint32_t(g);
    }
}

// ------------------------------------------------------------------ emit
// Block sums of the tile counts taken in depth order.
__global__ void __launch_bounds__(T)
emit_upsweep(const uint32_t *__restrict__ sorted_gid, const uint32_t *__restrict__ tcount,
             const uint32_t *__restrict__ d_n, uint32_t *__restrict__ blocksum) {
    __shared__ uint32_t s_w[WARPS];
    const uint32_t n = *d_n;
    uint32_t t0, t1;
    block_tiles(n, blockIdx.x, gridDim.x, t0, t1);
    const uint32_t end = min(n, t1 * TILE);
    uint32_t s = 0;
    for (uint32_t i = t0 * TILE + threadIdx.x; i < end; i += T) s += tcount[sorted_gid[i]];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) s_w[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t t = 0;
        for (int w = 0; w < WARPS; ++w) t += s_w[w];
        blocksum[blockIdx.x] = t;
    }
}

// Scan of the block sums; writes the intersection count and the capacity check.
__global__ void __launch_bounds__(1024)
emit_scan(uint32_t *blocksum, int nblocks, uint32_t *counters, uint32_t capacity) {
    __shared__ uint32_t s_total;
    cta_exclusive_scan(blocksum, nblocks, &s_total);
    __syncthreads();
    if (threadIdx.x == 0) {
        const uint32_t x = s_total;
        counters[CNT_ISECT] = x;
        if (x > capacity) {
            counters[CNT_STATUS] = QR_ERR_CAPACITY;
            counters[CNT_SORT_N] = 0;
        } else {
            counters[CNT_SORT_N] = x;
        }
    }
}

// Per-Gaussian exclusive offsets of the intersection list, in depth order.
__global__ void __launch_bounds__(T)
emit_offsets(const uint32_t *__restrict__ sorted_gid, const uint32_t *__restrict__ tcount,
             const uint32_t *__restrict__ d_n, const uint32_t *__restrict__ blocksum,
             uint32_t *__restrict__ off) {
    __shared__ uint32_t s_w[32];
    const uint32_t n = *d_n;
    uint32_t t0, t1;
    block_tiles(n, blockIdx.x, gridDim.x, t0, t1);
    const uint32_t end = min(n, t1 * TILE);
    uint32_t run = blocksum[blockIdx.x];
    for (uint32_t base = t0 * TILE; base < end; base += T) {
        const uint32_t i = base + threadIdx.x;
        const uint32_t c = i < end ? tcount[sorted_gid[i]] : 0u;
        uint32_t tot;
        const uint32_t inc = block_inclusive_scan(c, s_w, tot);
        if (i < end) off[i] = run + inc - c;
        run += tot;
    }
}

// Last index s in [0, n) with off[s] <= target (off[0] == 0 <= target), found
// by one warp with 32-way splits.
__device__ __forceinline__ uint32_t warp_upper_index(const uint32_t *off, uint32_t n, uint32_t target) {
    const int lane = threadIdx.x & 31;
    uint32_t lo = 0, hi = n;
    while (hi - lo > 32) {
        const uint32_t step = (hi - lo + 31) / 32;
        const uint32_t pos = lo + lane * step;
        const bool le = pos < hi && off[pos] <= target;
        const int k = __popc(__ballot_sync(0xffffffffu, le));
        lo = lo + (k - 1) * step;
        hi = min(hi, lo + step);
    }
    const uint32_t pos = lo + lane;
    const bool le = pos < hi && off[pos] <= target;
    return lo + __popc(__ballot_sync(0xffffffffu, le)) - 1;
}

// Load-balanced expansion: each CTA owns EMIT_CHUNK consecutive output slots,
// finds the Gaussians that own them, and writes one (tile, id) pair per slot
// with coalesced stores.  Work per CTA is independent of footprint sizes.
constexpr int EMIT_CHUNK = 2048;
__global__ void __launch_bounds__(T)
emit_expand(const uint32_t *__restrict__ off, const uint32_t *__restrict__ sorted_gid,
            const uint2 *__restrict__ rect, const uint32_t *__restrict__ d_n,
            const uint32_t *__restrict__ counters, int tiles_x, uint32_t *__restrict__ ikey,
            uint32_t *__restrict__ ival) {
    __shared__ uint32_t s_off[EMIT_CHUNK + 1];
    __shared__ uint32_t s_gid[EMIT_CHUNK + 1];
    __shared__ uint2 s_rect[EMIT_CHUNK + 1];
    __shared__ uint32_t s_range[2];
    const uint32_t X = counters[CNT_SORT_N];   // 0 when the capacity was exceeded
    const uint32_t n = *d_n;
    for (uint32_t o0 = blockIdx.x * uint32_t(EMIT_CHUNK); o0 < X; o0 += gridDim.x * uint32_t(EMIT_CHUNK)) {
        const uint32_t o1 = min(X, o0 + uint32_t(EMIT_CHUNK));
        if (threadIdx.x < 32) {
            const uint32_t s0 = warp_upper_index(off, n, o0);
            const uint32_t s1 = warp_upper_index(off, n, o1 - 1);
            if (threadIdx.x == 0) { s_range[0] = s0; s_range[1] = s1; }
        }
        __syncthreads();
        const uint32_t s0 = s_range[0], len = s_range[1] - s_range[0] + 1;   // <= EMIT_CHUNK
        for (uint32_t i = threadIdx.x; i < len; i += T) {
            const uint32_t g = sorted_gid[s0 + i];
            s_off[i] = off[s0 + i];
            s_gid[i] = g;
            s_rect[i] = rect[g];
        }
        __syncthreads();
        for (uint32_t o = o0 + threadIdx.x; o < o1; o += T) {
            uint32_t lo = 0, hi = len;             // last local index with s_off <= o
            while (hi - lo > 1) {
                const uint32_t mid = (lo + hi) >> 1;
                if (s_off[mid] <= o) lo = mid; else hi = mid;
            }
            const uint2 rc = s_rect[lo];
            const uint32_t tx0 = rc.x & 0xFFFFu, ty0 = rc.x >> 16, tx1 = rc.y & 0xFFFFu;
            const uint32_t wx = tx1 - tx0 + 1, j = o - s_off[lo];
            ikey[o] = (ty0 + j / wx) * uint32_t(tiles_x) + tx0 + j % wx;
            ival[o] = s_gid[lo];
        }
        __syncthreads();
    }
}

// ------------------------------------------------------------------ ranges
__global__ void __launch_bounds__(T)
tile_ranges(const uint32_t *__restrict__ ikey, const uint32_t *__restrict__ counters,
            uint2 *__restrict__ ranges) {
    const uint32_t n = counters[CNT_SORT_N];
    for (uint32_t i = blockIdx.x * T + threadIdx.x; i < n; i += gridDim.x * T) {
        const uint32_t t = ikey[i];
        if (i == 0 || ikey[i - 1] != t) ranges[t].x = i;
        if (i + 1 == n || ikey[i + 1] != t) ranges[t].y = i + 1;
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

int tile_bits_for(int tiles) {
    int b = 1;
    while ((1 << b) < tiles) ++b;
    return b;
}

cudaError_t launch_sort(const qr_frame &f, cudaStream_t s) {
    uint32_t *counters = slot<uint32_t>(f, S_COUNTERS);
    uint32_t *hist = slot<uint32_t>(f, S_HIST);
    uint32_t *digitsum = slot<uint32_t>(f, S_DIGITSUM);
    const int tiles = num_tiles(f);
    cudaError_t e = cudaMemsetAsync(slot<uint2>(f, S_RANGES), 0, sizeof(uint2) * size_t(tiles), s);
    if (e != cudaSuccess) return e;
    if (f.n == 0) return cudaSuccess;
    // 0. pack the kept Gaussians (id order) -> counters[CNT_VISIBLE] items
    const int nblk = int((f.n + kProjectThreads - 1) / kProjectThreads);
    uint32_t *viscnt = slot<uint32_t>(f, S_VISCNT);
    compact_scan<<<1, 1024, 0, s>>>(viscnt, nblk, counters);
    compact_scatter<<<nblk, kProjectThreads, 0, s>>>(slot<uint32_t>(f, S_GKEY), viscnt, f.n,
                                                     slot<uint32_t>(f, S_DKEY0),
                                                     slot<uint32_t>(f, S_DVAL0));
    count_launch(2);
    // 1. depth sort of the kept Gaussians
    const int nb_depth = sort_blocks_for(f.n);
    int in_b = 0;
    e = radix_sort_pairs(slot<uint32_t>(f, S_DKEY0), slot<uint32_t>(f, S_DVAL0),
                         slot<uint32_t>(f, S_DKEY1), slot<uint32_t>(f, S_DVAL1),
                         counters + CNT_VISIBLE, f.n, 0, 32, hist, digitsum, nb_depth, &in_b, s);
    if (e != cudaSuccess) return e;
    const uint32_t *sorted_gid = slot<uint32_t>(f, in_b ? S_DVAL1 : S_DVAL0);
    // 2. scan of tile counts in depth order + emit
    uint32_t *blocksum = slot<uint32_t>(f, S_BLOCKSUM);
    uint32_t *offs = slot<uint32_t>(f, in_b ? S_DKEY0 : S_DKEY1);  // the free key buffer
    int dev = 0, sms = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    emit_upsweep<<<nb_depth, T, 0, s>>>(sorted_gid, slot<uint32_t>(f, S_TCOUNT),
                                        counters + CNT_VISIBLE, blocksum);
    emit_scan<<<1, 1024, 0, s>>>(blocksum, nb_depth, counters, uint32_t(f.max_isect));
    emit_offsets<<<nb_depth, T, 0, s>>>(sorted_gid, slot<uint32_t>(f, S_TCOUNT),
                                        counters + CNT_VISIBLE, blocksum, offs);
    emit_expand<<<sms * 2, T, 0, s>>>(offs, sorted_gid, slot<uint2>(f, S_RECT),
                                      counters + CNT_VISIBLE, counters, f.tiles_x,
                                      slot<uint32_t>(f, S_IKEY0), slot<uint32_t>(f, S_IVAL0));
    count_launch(4);
    // 3. stable sort of the intersections by tile id
    int ib = 0;
    e = radix_sort_pairs(slot<uint32_t>(f, S_IKEY0), slot<uint32_t>(f, S_IVAL0),
                         slot<uint32_t>(f, S_IKEY1), slot<uint32_t>(f, S_IVAL1),
                         counters + CNT_SORT_N, f.max_isect, 0, tile_bits_for(tiles), hist,
                         digitsum, f.sort_blocks, &ib, s);
    if (e != cudaSuccess) return e;
    // 4. tile ranges
    const uint32_t *ikey = slot<uint32_t>(f, ib ? S_IKEY1 : S_IKEY0);
    tile_ranges<<<sms * 4, T, 0, s>>>(ikey, counters, slot<uint2>(f, S_RANGES));
    count_launch();
    return cudaGetLastError();
}

}  // namespace qr
