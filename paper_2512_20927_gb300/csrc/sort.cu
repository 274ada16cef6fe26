// K2-K4: binning, per-tile depth sort and tile ranges (Sec. 3 "tiling
// strategy"; the depth-ordered index list I of each ray, Sec. 4.2).
//
// Result: for every screen tile, the ids of the Gaussians whose footprint
// touches it, ordered by (camera depth, id) -- the order a stable sort of
// 64-bit (tile << 32 | depth) keys over id-ordered input gives.
//
// GB300 design (4 kernels after the projection, no global depth sort):
//   1. the projection (K1) counts, per 256 consecutive ids, the kept
//      Gaussians and the sum of their tile counts;
//   2. bin_scan (one CTA) scans the per-256-id counts (first output slot of
//      each kept Gaussian's block, totals, capacity check) and integrates the
//      2-D difference array of per-tile counts that the projection filled
//      (4 atomics per kept Gaussian instead of one per intersection) into
//      per-tile counts and exclusive offsets, i.e. the tile ranges;
//   3. offsets_apply compacts the kept Gaussians (id order) and gives each
//      its first output slot; offsets of kept Gaussians are strictly
//      increasing;
//   4. expand_scatter: a load-balanced expansion -- each CTA owns 1024
//      consecutive output slots, stages their owners (the kept Gaussians from
//      the owner of the chunk's first slot, which offsets_apply recorded, to
//      the owner of the next chunk's first slot), derives each slot's tile from
//      the owner's footprint rectangle, and writes (depth << 32 | id) into
//      its tile's bucket at an atomically claimed position (counted per tile
//      in shared memory first, one global atomic per touched tile, when the
//      grid has at most 4096 tiles);
//   5. tile_sort: one CTA per tile sorts a bucket of up to 2048 keys
//      (bitonic network over the unique 64-bit keys in registers: register
//      swaps, warp shuffles, shared memory only for the cross-warp strides)
//      and writes the ids; a larger bucket goes to a list, which
//      tile_sort_big's persistent CTAs of 1024 threads work through: up to
//      8192 keys merge-sorted in shared memory (runs of 8 in registers, then
//      merge-path rounds between two buffers), beyond that in 8192-key
//      chunks merged in global memory by the same CTA, so no size is refused.
// Keys are unique, so the order inside a bucket before step 5 does not matter
// and the result is deterministic.  No CTA waits for another.  Counts live in
// device memory, so the stage can be captured in a CUDA graph.
#include "qr_internal.cuh"

namespace qr {
namespace {

constexpr int T = 256;
constexpr int EMIT_CHUNK = kEmitChunk;
constexpr int TB = 1024;                 // threads of the big-bucket sort
constexpr int BIG_CAP = 8192;            // keys a big bucket sorts in shared memory (2 x 68 KB)
constexpr int BIG_SLOTS = BIG_CAP + BIG_CAP / 16;   // with one pad word per 16 keys
constexpr int kScanSmemTiles = 48 * 1024; // tile counts bin_scan integrates in shared memory
constexpr int kAggTiles = 4096;           // tile grids whose bucket claims are aggregated per CTA

// ------------------------------------------------------------------ offsets
// Compacted kept ids (id order) and their first output slots.
// It also records, for every expansion chunk, the kept index that owns the
// chunk's first slot (chunks past `nchunk` -- a capacity overflow -- are
// not recorded; the expansion then has nothing to do).
__global__ void __launch_bounds__(kProjectThreads)
offsets_apply(const uint32_t *__restrict__ tcount, const uint32_t *__restrict__ kept_base,
              const uint32_t *__restrict__ tsum_base, int64_t n, uint32_t *__restrict__ kid,
              uint32_t *__restrict__ koff, uint32_t *__restrict__ chunk_owner, uint32_t nchunk) {
    pdl_wait();   // the predecessor's outputs are complete and visible
    __shared__ uint32_t s_w[32];
    const int64_t g = int64_t(blockIdx.x) * kProjectThreads + threadIdx.x;
    const uint32_t c = g < n ? tcount[g] : 0u;
    const uint32_t k = c > 0 ? 1u : 0u;
    uint32_t tot;
    const uint32_t kinc = block_inclusive_scan(k, s_w, tot);
    const uint32_t cinc = block_inclusive_scan(c, s_w, tot);
    if (k) {
        const uint32_t slot = kept_base[blockIdx.x] + kinc - 1u;
        const uint32_t a = tsum_base[blockIdx.x] + cinc - c;
        kid[slot] = uint32_t(g);
        koff[slot] = a;
        for (uint32_t ch = (a + EMIT_CHUNK - 1) / EMIT_CHUNK; ch < nchunk && ch * EMIT_CHUNK < a + c; ++ch)
            chunk_owner[ch] = slot;
    }
}

// Owners of the slots [o0, o1) staged in shared memory: kept indices s0 (the
// owner of o0, recorded by offsets_apply) .. s1 (the owner of the next
// chunk's first slot, or the last kept Gaussian), at most EMIT_CHUNK + 1.
struct ExpandSmem {
    uint32_t off[EMIT_CHUNK + 1];
    uint32_t gid[EMIT_CHUNK + 1];
    uint32_t key[EMIT_CHUNK + 1];
    uint2 rect[EMIT_CHUNK + 1];
};

__device__ __forceinline__ uint32_t stage_owners(ExpandSmem &sm, const uint32_t *koff,
                                                 const uint32_t *kid, const uint2 *rect,
                                                 const uint32_t *gkey, uint32_t s0, uint32_t s1) {
    const uint32_t len = s1 - s0 + 1;
    for (uint32_t i = threadIdx.x; i < len; i += T) {
        const uint32_t g = kid[s0 + i];
        sm.off[i] = koff[s0 + i];
        sm.gid[i] = g;
        sm.key[i] = gkey[g];
        sm.rect[i] = rect[g];
    }
    __syncthreads();
    return len;
}

__device__ __forceinline__ void slot_owner(const ExpandSmem &sm, uint32_t len, uint32_t o,
                                           int tiles_x, uint32_t &g, uint32_t &tile,
                                           uint32_t &key) {
    uint32_t lo = 0, hi = len;
    while (hi - lo > 1) {
        const uint32_t mid = (lo + hi) >> 1;
        if (sm.off[mid] <= o) lo = mid; else hi = mid;
    }
    const uint2 rc = sm.rect[lo];
    const uint32_t tx0 = rc.x & 0xFFFFu, ty0 = rc.x >> 16, tx1 = rc.y & 0xFFFFu;
    const uint32_t wx = tx1 - tx0 + 1, j = o - sm.off[lo];
    g = sm.gid[lo];
    key = sm.key[lo];
    tile = (ty0 + j / wx) * uint32_t(tiles_x) + tx0 + j % wx;
}

// One CTA: exclusive scans of the per-256-id kept counts and tile sums (the
// kept Gaussians' first output slots, totals, capacity check), then the tile
// counts from the difference array (prefix sums along x, then y) and their
// exclusive offsets, i.e. the tile ranges; the counts become zeroed cursors.
// The counts are integrated in shared memory when the tile grid fits (up to
// kScanSmemTiles tiles, e.g. 4K frames with 16x16 tiles), else in the cursor
// array itself.  Rows are summed by one warp each (shuffle scans), columns by
// one thread each.  Partial sums may be negative; the uint32 arithmetic is
// exact modulo 2^32 and the integrated counts are not.
__global__ void __launch_bounds__(1024)
bin_scan(uint32_t *kept, uint32_t *tsum, int nblk, uint32_t *counters, uint32_t capacity,
         const int *__restrict__ diff, uint32_t *tcnt, int tiles_x, int tiles_y, uint2 *ranges,
         int in_smem) {
    pdl_wait();   // the predecessor's outputs are complete and visible
    extern __shared__ uint32_t s_cnt[];
    __shared__ uint32_t s_w[64];
    // both per-block scans in one pass, each thread owning `per` consecutive blocks
    const int per = (nblk + int(blockDim.x) - 1) / int(blockDim.x);
    const int b0 = int(threadIdx.x) * per;
    uint2 own = make_uint2(0u, 0u);
    for (int i = 0; i < per; ++i) {
        const int bb = b0 + i;
        if (bb < nblk) { own.x += kept[bb]; own.y += tsum[bb]; }
    }
    uint2 tot;
    const uint2 inc = block_inclusive_scan2(own, s_w, tot);
    uint2 ex = make_uint2(inc.x - own.x, inc.y - own.y);
    for (int i = 0; i < per; ++i) {
        const int bb = b0 + i;
        if (bb < nblk) {
            const uint32_t k = kept[bb], t = tsum[bb];
            kept[bb] = ex.x;
            tsum[bb] = ex.y;
            ex.x += k;
            ex.y += t;
        }
    }
    const uint32_t isect = tot.y;
    const bool over = isect > capacity;
    if (threadIdx.x == 0) {
        counters[CNT_BIG] = 0u;
        counters[CNT_VISIBLE] = tot.x;
        counters[CNT_ISECT] = isect;
        if (over) counters[CNT_STATUS] = QR_ERR_CAPACITY;
        counters[CNT_SORT_N] = over ? 0u : isect;
    }
    const int stride = tiles_x + 1;
    const int tiles = tiles_x * tiles_y;
    if (over) {   // capacity exceeded: every tile list is empty
        for (int t = threadIdx.x; t < tiles; t += blockDim.x) {
            ranges[t] = make_uint2(0u, 0u);
            tcnt[t] = 0u;
        }
        return;
    }
    uint32_t *A = in_smem ? s_cnt : tcnt;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarps = blockDim.x >> 5;
    for (int y = warp; y < tiles_y; y += nwarps) {
        uint32_t carry = 0;
        for (int x0 = 0; x0 < tiles_x; x0 += 32) {
            const int x = x0 + lane;
            uint32_t v = 0u;
            if (x < tiles_x)
#pragma unroll
                for (int r = 0; r < kDiffCopies; ++r)
                    v += uint32_t(diff[size_t(r) * stride * (tiles_y + 1) + y * stride + x]);
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t t = __shfl_up_sync(0xffffffffu, v, o);
                if (lane >= o) v += t;
            }
            if (x < tiles_x) A[y * tiles_x + x] = carry + v;
            carry += __shfl_sync(0xffffffffu, v, 31);
        }
    }
    __syncthreads();
    for (int x = threadIdx.x; x < tiles_x; x += blockDim.x) {
        uint32_t run = 0;
        for (int y = 0; y < tiles_y; ++y) {
            run += A[y * tiles_x + x];
            A[y * tiles_x + x] = run;
        }
    }
    __syncthreads();
    uint32_t carry = 0;
    for (int base = 0; base < tiles; base += blockDim.x) {
        const int t = base + threadIdx.x;
        const uint32_t c = t < tiles ? A[t] : 0u;
        uint32_t chunk;
        const uint32_t inc = block_inclusive_scan(c, s_w, chunk);
        if (t < tiles) ranges[t] = make_uint2(carry + inc - c, carry + inc);
        carry += chunk;
    }
    __syncthreads();
    for (int t = threadIdx.x; t < tiles; t += blockDim.x) tcnt[t] = 0u;
}

// AGG: tile grids of at most kAggTiles tiles claim bucket positions per CTA:
// shared-memory atomics count the chunk's slots per tile (and give each slot
// its rank), then one global atomic per touched tile reserves the chunk's
// run in the bucket.  Otherwise every warp claims with one global atomic per
// distinct tile among its 32 slots.
template <bool AGG>
__global__ void __launch_bounds__(T)
expand_scatter(const uint32_t *__restrict__ koff, const uint32_t *__restrict__ kid,
               const uint2 *__restrict__ rect, const uint32_t *__restrict__ gkey,
               const uint32_t *__restrict__ chunk_owner, const uint32_t *__restrict__ counters,
               int tiles_x, int tiles, const uint2 *__restrict__ ranges,
               uint32_t *__restrict__ cursor, unsigned long long *__restrict__ keys) {
    pdl_wait();   // the predecessor's outputs are complete and visible
    __shared__ ExpandSmem sm;
    extern __shared__ uint32_t s_agg[];   // AGG: [tiles] counts, [tiles] run bases
    const uint32_t X = counters[CNT_SORT_N];
    const uint32_t nk = counters[CNT_VISIBLE];
    const int lane = threadIdx.x & 31;
    constexpr int PER = EMIT_CHUNK / T;
    for (uint32_t c = blockIdx.x; c * uint32_t(EMIT_CHUNK) < X; c += gridDim.x) {
        const uint32_t o0 = c * uint32_t(EMIT_CHUNK);
        const uint32_t o1 = min(X, o0 + uint32_t(EMIT_CHUNK));
        if (AGG)
            for (int t = threadIdx.x; t < tiles; t += T) s_agg[t] = 0u;
        const uint32_t s0 = chunk_owner[c];
        const uint32_t s1 = o1 < X ? chunk_owner[c + 1] : nk - 1u;
        const uint32_t len = stage_owners(sm, koff, kid, rect, gkey, s0, s1);   // ends with a barrier
        if (AGG) {
            uint32_t tl[PER], gg[PER], kk[PER], rk[PER];
#pragma unroll
            for (int k = 0; k < PER; ++k) {
                const uint32_t o = o0 + threadIdx.x + k * T;
                tl[k] = 0xFFFFFFFFu;
                if (o < o1) {
                    slot_owner(sm, len, o, tiles_x, gg[k], tl[k], kk[k]);
                    rk[k] = atomicAdd(&s_agg[tl[k]], 1u);
                }
            }
            __syncthreads();
            for (int t = threadIdx.x; t < tiles; t += T) {
                const uint32_t cnt = s_agg[t];
                if (cnt) s_agg[tiles + t] = atomicAdd(&cursor[t], cnt);
            }
            __syncthreads();
#pragma unroll
            for (int k = 0; k < PER; ++k) {
                if (tl[k] == 0xFFFFFFFFu) continue;
                keys[ranges[tl[k]].x + s_agg[tiles + tl[k]] + rk[k]] =
                    (static_cast<unsigned long long>(kk[k]) << 32) | gg[k];
            }
        } else {
            for (uint32_t base = o0; base < o1; base += T) {
                const uint32_t o = base + threadIdx.x;
                uint32_t g = 0, tile = 0xFFFFFFFFu, key = 0;
                if (o < o1) slot_owner(sm, len, o, tiles_x, g, tile, key);
                const unsigned peers = __match_any_sync(0xffffffffu, tile);
                const int leader = __ffs(peers) - 1;
                uint32_t pos = 0;
                if (o < o1 && lane == leader) pos = atomicAdd(&cursor[tile], uint32_t(__popc(peers)));
                pos = __shfl_sync(0xffffffffu, pos, leader);
                if (o < o1) {
                    const uint32_t rank = __popc(peers & ((1u << lane) - 1u));
                    keys[ranges[tile].x + pos + rank] = (static_cast<unsigned long long>(key) << 32) | g;
                }
            }
        }
        __syncthreads();
    }
}

// ------------------------------------------------------------------ per-tile sort
// A bucket of up to NTH*E keys, loaded E per thread in blocked order and
// padded with ~0, sorted by the register bitonic network, ids written out.
template <int E, int NTH = T>
__device__ void sort_registers(const unsigned long long *__restrict__ src, int n,
                               unsigned long long *s, uint32_t *__restrict__ dst) {
    const int base = threadIdx.x * E;
    unsigned long long v[E];
#pragma unroll
    for (int e = 0; e < E; ++e) v[e] = base + e < n ? src[base + e] : ~0ull;
    bitonic_regs<E, NTH, unsigned long long>(v, s);
#pragma unroll
    for (int e = 0; e < E; ++e)
        if (base + e < n) dst[base + e] = uint32_t(v[e]);
}

// Merge sorted A[0,na) and B[0,nb) into C with the whole CTA of NT threads
// (merge path).
template <int NT>
__device__ __forceinline__ void merge_cta(const unsigned long long *A, int na,
                                          const unsigned long long *B, int nb,
                                          unsigned long long *C) {
    const int total = na + nb;
    const int per = (total + NT - 1) / NT;
    const int d0 = min(total, int(threadIdx.x) * per), d1 = min(total, d0 + per);
    auto split = [&](int d) {
        int lo = max(0, d - nb), hi = min(d, na);
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (A[mid] <= B[d - 1 - mid]) lo = mid + 1; else hi = mid;
        }
        return lo;
    };
    int i = split(d0), j = d0 - i;
    const int iend = split(d1), jend = d1 - iend;
    for (int d = d0; d < d1; ++d) {
        if (i < iend && (j >= jend || A[i] <= B[j])) C[d] = A[i++];
        else C[d] = B[j++];
    }
}

// Buckets of up to 8 T keys (registers, up to 8 per thread).  A larger
// bucket is appended to the list of big buckets that tile_sort_big works
// through, so its register and shared-memory needs do not lower this
// kernel's occupancy for every tile.
__global__ void __launch_bounds__(T)
tile_sort(const uint2 *__restrict__ ranges, unsigned long long *__restrict__ keys,
          uint32_t *__restrict__ igid, uint32_t *__restrict__ big, uint32_t *__restrict__ counters) {
    pdl_wait();   // the predecessor's outputs are complete and visible
    __shared__ unsigned long long s_k[8 * T];
    const uint2 r = ranges[blockIdx.x];
    const int n = int(r.y - r.x);
    if (n > 8 * T) {
        if (threadIdx.x == 0) big[atomicAdd(&counters[CNT_BIG], 1u)] = blockIdx.x;
        return;
    }
    if (n == 0) return;
    unsigned long long *src = keys + r.x;
    if (n <= 2 * T) {
        if (n <= T) sort_registers<1>(src, n, s_k, igid + r.x);
        else sort_registers<2>(src, n, s_k, igid + r.x);
        return;
    }
    if (n <= 4 * T) sort_registers<4>(src, n, s_k, igid + r.x);
    else sort_registers<8>(src, n, s_k, igid + r.x);
}

// ------------------------------------------------------------------ big buckets
// Eight keys in registers sorted by Batcher's odd-even merge network (19
// compare-exchanges).
__device__ __forceinline__ void cx(unsigned long long &a, unsigned long long &b) {
    const unsigned long long lo = a < b ? a : b, hi = a < b ? b : a;
    a = lo;
    b = hi;
}
__device__ __forceinline__ void sort8(unsigned long long (&v)[8]) {
    cx(v[0], v[1]); cx(v[2], v[3]); cx(v[4], v[5]); cx(v[6], v[7]);
    cx(v[0], v[2]); cx(v[1], v[3]); cx(v[4], v[6]); cx(v[5], v[7]);
    cx(v[1], v[2]); cx(v[5], v[6]);
    cx(v[0], v[4]); cx(v[1], v[5]); cx(v[2], v[6]); cx(v[3], v[7]);
    cx(v[2], v[4]); cx(v[3], v[5]);
    cx(v[1], v[2]); cx(v[3], v[4]); cx(v[5], v[6]);
}

// Shared-memory slot of key i in a big-bucket buffer: one pad word after
// every 16 keys.  Threads that own E consecutive keys (E = 2..16) then touch
// 16 different bank pairs per half-warp instead of 16 / E.
__device__ __forceinline__ int pad(int i) { return i + (i >> 4); }

// Sort n <= TB * E unique keys in shared memory (padded slots): runs of 8
// sorted in registers, then merge rounds of doubling run length L between the
// two buffers s and t.  In a round thread i produces outputs [iE, iE + E) of
// its pair of runs (2L is a multiple of E, so the range never crosses pairs):
// a merge-path binary search gives its start in each run and the E outputs
// are merged straight into the other buffer.  Returns the buffer holding the
// sorted keys.
template <int E>
__device__ unsigned long long *sort_smem(unsigned long long *s, unsigned long long *t, int n) {
    for (int r0 = int(threadIdx.x) * 8; r0 < n; r0 += TB * 8) {
        unsigned long long v[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) v[e] = r0 + e < n ? s[pad(r0 + e)] : ~0ull;
        sort8(v);
#pragma unroll
        for (int e = 0; e < 8; ++e)
            if (r0 + e < n) s[pad(r0 + e)] = v[e];
    }
    __syncthreads();
    const int d0 = int(threadIdx.x) * E;
    const int m = max(0, min(E, n - d0));
    for (int L = 8; L < n; L <<= 1) {
        if (m > 0) {
            const int ps = d0 & ~(2 * L - 1);
            const int na = min(L, n - ps);
            const int nb = max(0, min(L, n - ps - na));
            const int pb = ps + na;   // run A is keys [ps, pb), run B [pb, pb + nb)
            const int diag = d0 - ps;
            int lo = max(0, diag - nb), hi = min(diag, na);
            while (lo < hi) {
                const int mid = (lo + hi) >> 1;
                if (s[pad(ps + mid)] < s[pad(pb + diag - 1 - mid)]) lo = mid + 1; else hi = mid;
            }
            int i = lo, j = diag - lo;
            for (int e = 0; e < m; ++e) {
                const unsigned long long ka = i < na ? s[pad(ps + i)] : ~0ull;
                const unsigned long long kb = j < nb ? s[pad(pb + j)] : ~0ull;
                const bool take_a = j >= nb || (i < na && ka < kb);
                t[pad(d0 + e)] = take_a ? ka : kb;
                i += take_a ? 1 : 0;
                j += take_a ? 0 : 1;
            }
        }
        // Thread i writes keys [iE, iE + E) in every round, and the next round
        // (run length 2L) reads only the aligned block of 4L keys holding its
        // outputs.  While 4L <= 32 E that block is one warp's own outputs (and
        // was read by that warp alone in this round), so the warp's barrier
        // orders it; the last round's outputs are read by every thread.
        if (4 * L <= 32 * E && 2 * L < n) __syncwarp();
        else __syncthreads();
        unsigned long long *x = s;
        s = t;
        t = x;
    }
    return s;
}

__device__ __forceinline__ unsigned long long *sort_smem_any(unsigned long long *s,
                                                             unsigned long long *t, int n) {
    if (n <= TB * 2) return sort_smem<2>(s, t, n);
    if (n <= TB * 4) return sort_smem<4>(s, t, n);
    return sort_smem<8>(s, t, n);
}

// The buckets of more than 8 T keys, listed by tile_sort: persistent CTAs of
// TB threads (one per SM: 136 KB of shared memory) take them in turn.  Up to
// BIG_CAP keys are merge-sorted in shared memory (faster here than the
// register bitonic network over 1024 threads: 232 vs 365 us for the object
// frame's sort stage); a larger bucket is sorted in BIG_CAP chunks whose
// sorted runs are merged in global memory by the same CTA (merge path,
// ping-ponging between the key buffer and the scratch buffer), so no size is
// refused.
__global__ void __launch_bounds__(TB, 1)
tile_sort_big(const uint2 *__restrict__ ranges, unsigned long long *__restrict__ keys,
              unsigned long long *__restrict__ scratch, uint32_t *__restrict__ igid,
              const uint32_t *__restrict__ big, const uint32_t *__restrict__ counters) {
    pdl_wait();   // the predecessor's outputs are complete and visible
    extern __shared__ unsigned long long s_k[];   // 2 x BIG_SLOTS (padded slots)
    unsigned long long *s_t = s_k + BIG_SLOTS;
    const uint32_t nbig = counters[CNT_BIG];
    for (uint32_t bi = blockIdx.x; bi < nbig; bi += gridDim.x) {
        const uint2 r = ranges[big[bi]];
        const int n = int(r.y - r.x);
        unsigned long long *src = keys + r.x;
        if (n <= BIG_CAP) {
            for (int i = threadIdx.x; i < n; i += TB) s_k[pad(i)] = src[i];
            __syncthreads();
            const unsigned long long *o = sort_smem_any(s_k, s_t, n);
            for (int i = threadIdx.x; i < n; i += TB) igid[r.x + i] = uint32_t(o[pad(i)]);
            __syncthreads();
            continue;
        }
        for (int c0 = 0; c0 < n; c0 += BIG_CAP) {
            const int m = min(BIG_CAP, n - c0);
            for (int i = threadIdx.x; i < m; i += TB) s_k[pad(i)] = src[c0 + i];
            __syncthreads();
            const unsigned long long *o = sort_smem_any(s_k, s_t, m);
            for (int i = threadIdx.x; i < m; i += TB) src[c0 + i] = o[pad(i)];
            __syncthreads();
        }
        unsigned long long *a = src, *dst = scratch + r.x;
        for (int w = BIG_CAP; w < n; w <<= 1) {
            for (int a0 = 0; a0 < n; a0 += 2 * w) {
                const int na = min(w, n - a0);
                const int nb = min(w, n - a0 - na);
                merge_cta<TB>(a + a0, na, a + a0 + na, nb, dst + a0);
            }
            __syncthreads();
            unsigned long long *t = a;
            a = dst;
            dst = t;
        }
        for (int i = threadIdx.x; i < n; i += TB) igid[r.x + i] = uint32_t(a[i]);
        __syncthreads();
    }
}

}  // namespace

cudaError_t launch_sort(const qr_frame &f, cudaStream_t s) {
    uint32_t *counters = slot<uint32_t>(f, S_COUNTERS);
    const int tiles = num_tiles(f);
    uint2 *ranges = slot<uint2>(f, S_RANGES);
    uint32_t *tcnt = slot<uint32_t>(f, S_TCNT);
    int *diff = slot<int>(f, S_DIFF);
    cudaError_t e;
    if (f.n == 0) {   // nothing projected: empty tile lists
        e = cudaMemsetAsync(tcnt, 0, sizeof(uint32_t) * size_t(tiles), s);
        if (e == cudaSuccess) e = cudaMemsetAsync(ranges, 0, sizeof(uint2) * size_t(tiles), s);
        return e;
    }
    e = cudaFuncSetAttribute(tile_sort_big, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             int(2 * BIG_SLOTS * sizeof(unsigned long long)));
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int nblk = int((f.n + kProjectThreads - 1) / kProjectThreads);
    uint32_t *kept = slot<uint32_t>(f, S_VISCNT);
    uint32_t *tsum = slot<uint32_t>(f, S_BSUM);
    uint32_t *kid = slot<uint32_t>(f, S_KID);
    uint32_t *koff = slot<uint32_t>(f, S_OFF);
    const uint2 *rect = slot<uint2>(f, S_RECT);
    const int scan_smem = tiles <= kScanSmemTiles ? 1 : 0;
    const size_t scan_bytes = scan_smem ? sizeof(uint32_t) * size_t(tiles) : 0;
    e = cudaFuncSetAttribute(bin_scan, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             int(sizeof(uint32_t) * kScanSmemTiles));
    if (e != cudaSuccess) return e;
    e = pdl_launch(bin_scan, dim3(1), dim3(1024), scan_bytes, s, kept, tsum, nblk, counters,
                   uint32_t(f.max_isect), diff, tcnt, f.tiles_x, f.tiles_y, ranges, scan_smem);
    if (e != cudaSuccess) return e;
    uint32_t *chunk_owner = slot<uint32_t>(f, S_CHUNK);
    const uint32_t nchunk = uint32_t(f.max_isect / EMIT_CHUNK + 1);
    e = pdl_launch(offsets_apply, dim3(nblk), dim3(kProjectThreads), 0, s,
                   (const uint32_t *)slot<uint32_t>(f, S_TCOUNT), (const uint32_t *)kept,
                   (const uint32_t *)tsum, f.n, kid, koff, chunk_owner, nchunk);
    if (e != cudaSuccess) return e;
    auto *keys = slot<unsigned long long>(f, S_KEYS64);
    if (tiles <= kAggTiles) {
        const size_t agg = sizeof(uint32_t) * 2 * size_t(tiles);
        e = cudaFuncSetAttribute(expand_scatter<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 int(sizeof(uint32_t) * 2 * kAggTiles));
        if (e != cudaSuccess) return e;
        e = pdl_launch(expand_scatter<true>, dim3(sms * 4), dim3(T), agg, s, (const uint32_t *)koff,
                       (const uint32_t *)kid, rect, (const uint32_t *)slot<uint32_t>(f, S_GKEY),
                       (const uint32_t *)chunk_owner, counters, f.tiles_x, tiles, ranges, tcnt, keys);
    } else {
        e = pdl_launch(expand_scatter<false>, dim3(sms * 6), dim3(T), 0, s, (const uint32_t *)koff,
                       (const uint32_t *)kid, rect, (const uint32_t *)slot<uint32_t>(f, S_GKEY),
                       (const uint32_t *)chunk_owner, counters, f.tiles_x, tiles, ranges, tcnt, keys);
    }
    if (e != cudaSuccess) return e;
    // the per-tile cursors are dead once the keys are scattered: their slot
    // holds the list of big buckets
    e = pdl_launch(tile_sort, dim3(tiles), dim3(T), 0, s, (const uint2 *)ranges, keys,
                   slot<uint32_t>(f, S_IGID), tcnt, counters);
    if (e != cudaSuccess) return e;
    e = pdl_launch(tile_sort_big, dim3(unsigned(min(tiles, sms))), dim3(TB),
                   2 * BIG_SLOTS * sizeof(unsigned long long), s,
                   (const uint2 *)ranges, keys, slot<unsigned long long>(f, S_SCRATCH64),
                   slot<uint32_t>(f, S_IGID), (const uint32_t *)tcnt, (const uint32_t *)counters);
    count_launch(5);
    return e != cudaSuccess ? e : cudaGetLastError();
}

}  // namespace qr
