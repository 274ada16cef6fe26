// K8: open-vocabulary relevance (Sec. 5: cosine similarity of features and
// text embeddings), R[p][q] = sum_c map[p][c] * Q[q][c], on the 5th-generation
// tensor cores (tcgen05 / UMMA, FP32 accumulation in TMEM).  The map is the
// blend's FP32 output, so the product is memory-bound (~32 flops per byte of
// map at Q = 64): the kernels are built to stream the map at HBM speed.
//
// Main kernel (relevance_tma_kernel), when its shared memory fits:
//   * persistent, one CTA per SM, warp-specialised: warp 0 issues TMA
//     (cp.async.bulk.tensor) loads of 128-pixel x 32-channel FP32 map tiles
//     into a 4-stage ring in the 128-byte-swizzled K-major layout UMMA reads;
//   * warp 1 issues kind::tf32 UMMAs (TF32 keeps 10 mantissa bits of the map;
//     the BF16 queries are exact in TF32) into one of two TMEM accumulators
//     and commits each stage back to the producer through an mbarrier;
//   * warps 2-5 drain the other accumulator with tcgen05.ld and write FP32
//     rows of R while the next tile's MMAs run;
//   * the queries are staged once per CTA, converted to FP32 and swizzled.
// Fallback kernel (relevance_kernel), e.g. 128 queries of 512 channels whose
// FP32 copy would not fit next to the ring: persistent CTAs of 8 warps (two
// per SM) read each 128 x 64 FP32 slice with 16-byte streaming loads into
// registers one slice ahead, round to BF16 into a swizzled shared-memory stage
// and issue kind::f16 UMMAs.
// Every mbarrier wait is bounded; on timeout a CTA records
// QR_ERR_DEVICE_TIMEOUT in the status word, waits (bounded) for its own copies
// and MMAs, frees its TMEM and returns.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp8.h>

#include "qr_internal.cuh"
#include "tma.cuh"

namespace qr {
namespace {

constexpr int BM = 128;            // pixels per tile (TMEM lanes)
constexpr int BK = 64;             // channels per slice: 128 bytes of BF16
constexpr int NT = 256;            // threads (8 warps)
constexpr int PF = BM * 16 / NT;   // float4 of a 128 x 64 FP32 slice per thread
constexpr int A_STAGE = BM * BK * 2;   // 16 KB
constexpr unsigned kSpinLimit = 1u << 26;

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// K-major, 128-byte swizzle: row r of a 128-byte-wide slice, 16-byte chunk c.
__device__ __forceinline__ uint32_t swz(int r, int c) {
    return uint32_t(r) * 128u + uint32_t((c ^ (r & 7)) * 16);
}

// Shared-memory matrix descriptor (tcgen05): start >> 4, LBO (unused for
// swizzled K-major, 16 B), SBO = 1024 B between 8-row groups, fixed 0b001 at
// bit 46, swizzle mode 2 = 128 B at bits 61-63.
__device__ __forceinline__ uint64_t make_desc(uint32_t saddr) {
    return uint64_t((saddr & 0x3FFFFu) >> 4) | (uint64_t(1) << 16) | (uint64_t(1024 >> 4) << 32) |
           (uint64_t(1) << 46) | (uint64_t(2) << 61);
}

// Instruction descriptor, kind::f16: D = F32 (bits 4-5 = 1), A = B = BF16
// (bits 7-9, 10-12 = 1), both K-major, N >> 3 at bit 17, M >> 4 at bit 24.
__host__ __device__ constexpr uint32_t make_idesc(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | (uint32_t(N >> 3) << 17) | (uint32_t(M >> 4) << 24);
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(smem_u32(bar)), "r"(count) : "memory");
}

// Bounded wait for the phase with the given parity; false on timeout.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity) {
    const uint32_t a = smem_u32(bar);
    for (unsigned i = 0; i < kSpinLimit; ++i) {
        uint32_t done;
        asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
                     " selp.u32 %0, 1, 0, p;\n}\n"
                     : "=r"(done) : "r"(a), "r"(parity) : "memory");
        if (done) return true;
    }
    return false;
}

// The same decision for every thread of the CTA: thread 0 polls, all read the result.
__device__ __forceinline__ bool cta_wait(uint64_t *bar, uint32_t parity, int *s_flag) {
    if (threadIdx.x == 0) *s_flag = mbar_wait(bar, parity) ? 1 : 0;
    __syncthreads();
    const bool r = *s_flag != 0;
    __syncthreads();
    return r;
}

__device__ __forceinline__ void umma_bf16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc,
                                          uint32_t idesc, uint32_t accumulate) {
    asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                 " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n"
                 :: "r"(d_tmem), "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate) : "memory");
}

__device__ __forceinline__ void umma_commit(uint64_t *bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                 :: "r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ void tc_fence_before() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void fence_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// 16 consecutive accumulator columns of this warp's 32 TMEM lanes.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float *v) {
    uint32_t r[16];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 "
                 "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]),
                   "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]),
                   "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
                 : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// Issue the loads of an FP32 map slice (rows p0.., channels c0..c0+63) into
// registers: element i = threadIdx.x + k*NT is row i/16, float4 i%16, so a
// warp-wide load covers two rows with 256 contiguous bytes each.
__device__ __forceinline__ void fetch_slice(const float *__restrict__ map, int64_t P, int C,
                                            int64_t p0, int c0, float4 (&v)[PF]) {
#pragma unroll
    for (int k = 0; k < PF; ++k) {
        const int i = threadIdx.x + k * NT;
        const int64_t p = p0 + (i >> 4);
        v[k] = p < P ? __ldcs(reinterpret_cast<const float4 *>(map + p * C + c0 + (i & 15) * 4))
                     : make_float4(0.f, 0.f, 0.f, 0.f);
    }
}

// Round the fetched slice to BF16 into a 128-byte-swizzled K-major stage.
__device__ __forceinline__ void store_slice(const float4 (&v)[PF], unsigned char *stage) {
#pragma unroll
    for (int k = 0; k < PF; ++k) {
        const int i = threadIdx.x + k * NT;
        const int r = i >> 4, f4 = i & 15;
        const __nv_bfloat162 lo = __floats2bfloat162_rn(v[k].x, v[k].y);
        const __nv_bfloat162 hi = __floats2bfloat162_rn(v[k].z, v[k].w);
        uint2 packed;
        packed.x = *reinterpret_cast<const uint32_t *>(&lo);
        packed.y = *reinterpret_cast<const uint32_t *>(&hi);
        *reinterpret_cast<uint2 *>(stage + swz(r, f4 >> 1) + (f4 & 1) * 8) = packed;
    }
}

// ------------------------------------------------------------ TMA + TF32 path
// mbarrier arrive that also announces the bytes a TMA copy will deliver.
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;"
                 :: "r"(smem_u32(bar)), "r"(bytes) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" :: "r"(smem_u32(bar)) : "memory");
}

// 2-D tiled TMA load of box {32 floats, 128 rows} at (x = channel, y = pixel)
// into a 128-byte-swizzled shared-memory stage; completion is counted on bar.
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap *map, int x, int y,
                                            uint64_t *bar) {
    asm volatile("cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
                 " [%0], [%1, {%2, %3}], [%4];"
                 :: "r"(dst), "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y),
                    "r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ void umma_tf32(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc,
                                          uint32_t idesc, uint32_t accumulate) {
    asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                 " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n"
                 :: "r"(d_tmem), "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate) : "memory");
}

// Instruction descriptor, kind::tf32: D = F32 (bits 4-5 = 1), A = B = TF32
// (bits 7-9, 10-12 = 2), both K-major, N >> 3 at bit 17, M >> 4 at bit 24.
__host__ __device__ constexpr uint32_t make_idesc_tf32(int M, int N) {
    return (1u << 4) | (2u << 7) | (2u << 10) | (uint32_t(N >> 3) << 17) | (uint32_t(M >> 4) << 24);
}

// Bounded wait by one thread (at most `spin` polls); on timeout raises the
// CTA's abort flag.
__device__ __forceinline__ bool lane_wait(uint64_t *bar, uint32_t parity, volatile int *abort_flag,
                                          unsigned spin = kSpinLimit) {
    if (*abort_flag) return false;
    const uint32_t a = smem_u32(bar);
    for (unsigned i = 0; i < spin; ++i) {
        uint32_t done;
        asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
                     " selp.u32 %0, 1, 0, p;\n}\n"
                     : "=r"(done) : "r"(a), "r"(parity) : "memory");
        if (done) return true;
    }
    *abort_flag = 1;
    return false;
}

// Polls allowed to the first-level waits of the relevance kernels (those
// that set the abort flag); the drains after an abort keep kSpinLimit.
// Changed only through qr_set_wait_limit (a test hook).
unsigned g_wait_limit = kSpinLimit;

template <int QN>
__global__ void __launch_bounds__(NT, 2)
relevance_kernel(const float *__restrict__ map, const uint16_t *__restrict__ queries, int64_t P,
                 int C, float *__restrict__ out, int *__restrict__ status) {
    constexpr uint32_t TMEM_COLS = QN <= 32 ? 32 : QN <= 64 ? 64 : 128;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char *base = reinterpret_cast<unsigned char *>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    const int nslices = C / BK;
    unsigned char *sB = base;                                     // nslices x QN x 128 B
    unsigned char *sA = sB + size_t(nslices) * QN * 128;         // 2 stages x 16 KB
    uint64_t *bars = reinterpret_cast<uint64_t *>(sA + 2 * A_STAGE);   // 2 mbarriers
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(bars + 2);
    int *s_flag = reinterpret_cast<int *>(tmem_slot + 1);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    // queries -> swizzled K-major slices (16-byte chunks copied as they are)
    for (int i = threadIdx.x; i < nslices * QN * 8; i += NT) {
        const int s = i / (QN * 8), rem = i % (QN * 8), n = rem >> 3, c = rem & 7;
        const uint4 v = *reinterpret_cast<const uint4 *>(queries + size_t(n) * C + s * BK + c * 8);
        *reinterpret_cast<uint4 *>(sB + size_t(s) * QN * 128 + swz(n, c)) = v;
    }
    if (threadIdx.x == 0) {
        mbar_init(&bars[0], 1);
        mbar_init(&bars[1], 1);
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     :: "r"(smem_u32(tmem_slot)), "r"(TMEM_COLS) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    constexpr uint32_t idesc = make_idesc(BM, QN);
    uint32_t uses[2] = {0u, 0u};      // commits issued per stage
    bool ok = true;
    const int64_t tiles = (P + BM - 1) / BM;
    float4 regs[PF];
    if (int64_t(blockIdx.x) < tiles) fetch_slice(map, P, C, int64_t(blockIdx.x) * BM, 0, regs);
    for (int64_t t = blockIdx.x; t < tiles && ok; t += gridDim.x) {
        const int64_t p0 = t * BM;
        for (int s = 0; s < nslices; ++s) {
            const int st = s & 1;
            if (uses[st] > 0 && !cta_wait(&bars[st], (uses[st] - 1) & 1, s_flag)) { ok = false; break; }
            store_slice(regs, sA + st * A_STAGE);
            fence_async_smem();
            tc_fence_before();
            __syncthreads();
            tc_fence_after();
            if (threadIdx.x == 0) {
                const uint32_t a0 = smem_u32(sA + st * A_STAGE);
                const uint32_t b0 = smem_u32(sB + size_t(s) * QN * 128);
#pragma unroll
                for (int k = 0; k < BK / 16; ++k)
                    umma_bf16(tmem, make_desc(a0 + k * 32), make_desc(b0 + k * 32), idesc,
                              (s > 0 || k > 0) ? 1u : 0u);
                umma_commit(&bars[st]);
            }
            ++uses[st];
            // the next slice's loads fly while the tensor cores work on this one
            if (s + 1 < nslices) fetch_slice(map, P, C, p0, (s + 1) * BK, regs);
            else if (t + gridDim.x < tiles) fetch_slice(map, P, C, (t + gridDim.x) * BM, 0, regs);
        }
        if (!ok) break;
        // all MMAs of this tile are done once the last commit has landed
        const int last = (nslices - 1) & 1;
        if (!cta_wait(&bars[last], (uses[last] - 1) & 1, s_flag)) { ok = false; break; }
        tc_fence_after();
        // warp w reads TMEM lanes 32*(w%4).. (pixels) and half w/4 of the columns
        const int quarter = warp & 3, half = warp >> 2;
        constexpr int CW = QN >= 32 ? QN / 2 : QN;
        if (QN >= 32 || half == 0) {
            const int64_t p = p0 + quarter * 32 + lane;
            const uint32_t taddr = tmem + (uint32_t(quarter * 32) << 16);
#pragma unroll
            for (int c = half * CW; c < half * CW + CW; c += 16) {
                float v[16];
                tmem_ld16(taddr + uint32_t(c), v);
                if (p < P) {
                    float4 *o = reinterpret_cast<float4 *>(out + p * QN + c);
                    o[0] = make_float4(v[0], v[1], v[2], v[3]);
                    o[1] = make_float4(v[4], v[5], v[6], v[7]);
                    o[2] = make_float4(v[8], v[9], v[10], v[11]);
                    o[3] = make_float4(v[12], v[13], v[14], v[15]);
                }
            }
        }
        tc_fence_before();
        __syncthreads();
        tc_fence_after();
    }
    if (!ok && threadIdx.x == 0) atomicExch(status, int(QR_ERR_DEVICE_TIMEOUT));
    // a stage whose commit was not waited for may still be in flight: drain it
    for (int st = 0; st < 2; ++st)
        if (uses[st] > 0) cta_wait(&bars[st], (uses[st] - 1) & 1, s_flag);
    tc_fence_before();
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tmem), "r"(TMEM_COLS) : "memory");
}

constexpr int TT = 192;               // warp 0 TMA, warp 1 MMA, warps 2-5 epilogue
constexpr int STAGES = 4;             // FP32 map tiles in flight per CTA
constexpr int A_TILE = 128 * 32 * 4;  // 128 pixels x 32 channels FP32 = 16 KB

// Persistent, one CTA per SM, warp-specialised: a TMA producer streams
// 128 x 32 FP32 map tiles into a 4-stage 128-byte-swizzled ring, one thread
// issues kind::tf32 UMMAs (TF32 keeps 10 mantissa bits of the map, more than
// BF16) into one of two TMEM accumulators, and four epilogue warps drain the
// other accumulator with tcgen05.ld while the next tile's MMAs run.  The
// queries (BF16, exact in TF32) are staged once per CTA.  Every mbarrier wait
// is bounded; on timeout the CTA raises an abort flag, every role stops, the
// CTA waits (bounded) for its own TMA copies and MMAs, frees TMEM and reports
// QR_ERR_DEVICE_TIMEOUT.
template <int QN>
__global__ void __launch_bounds__(TT, 1)
relevance_tma_kernel(const __grid_constant__ CUtensorMap tmap, const uint16_t *__restrict__ queries,
                     int64_t P, int C, float *__restrict__ out, int *__restrict__ status,
                     unsigned spin) {
    constexpr uint32_t TMEM_COLS = 2 * QN < 32 ? 32 : 2 * QN;   // two accumulators
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char *base = reinterpret_cast<unsigned char *>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    const int nsl = C / 32;
    unsigned char *sA = base;                                       // STAGES x 16 KB
    unsigned char *sB = sA + STAGES * A_TILE;                       // nsl x QN x 128 B
    uint64_t *full = reinterpret_cast<uint64_t *>(sB + size_t(nsl) * QN * 128);
    uint64_t *empty = full + STAGES;
    uint64_t *tfull = empty + STAGES;
    uint64_t *tempty = tfull + 2;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(tempty + 2);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);
    uint32_t *s_count = reinterpret_cast<uint32_t *>(tmem_slot + 2);   // [0] TMA issued, [1] MMA slices
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    // queries -> FP32 in the K-major 128-byte-swizzled layout UMMA reads:
    // row n of slice s holds channels 32s .. 32s+31 in 16-byte chunks c ^ (n % 8)
    for (int i = threadIdx.x; i < QN * C; i += TT) {
        const int n = i / C, c = i - n * C;
        const int sl = c >> 5, cc = c & 31;
        const float v = __uint_as_float(uint32_t(queries[size_t(n) * C + c]) << 16);
        *reinterpret_cast<float *>(sB + size_t(sl) * QN * 128 + n * 128 +
                                   (((cc >> 2) ^ (n & 7)) << 4) + (cc & 3) * 4) = v;
    }
    if (threadIdx.x == 0) {
        for (int st = 0; st < STAGES; ++st) {
            mbar_init(&full[st], 1);
            mbar_init(&empty[st], 1);
        }
        for (int a = 0; a < 2; ++a) {
            mbar_init(&tfull[a], 1);
            mbar_init(&tempty[a], 4);
        }
        *abort_flag = 0;
        s_count[0] = s_count[1] = 0u;
        // make the initialised barriers visible to the TMA and tensor-core units
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     :: "r"(smem_u32(tmem_slot)), "r"(TMEM_COLS) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    const int64_t tiles = (P + 127) / 128;

    if (warp == 0 && lane == 0) {
        // TMA producer
        uint32_t it = 0;
        bool ok = true;
        for (int64_t t = blockIdx.x; t < tiles && ok; t += gridDim.x)
            for (int sl = 0; sl < nsl; ++sl) {
                const int st = int(it % STAGES);
                if (!lane_wait(&empty[st], ((it / STAGES) & 1u) ^ 1u, abort_flag, spin)) { ok = false; break; }
                mbar_expect_tx(&full[st], A_TILE);
                tma_load_2d(smem_u32(sA + st * A_TILE), &tmap, sl * 32, int(t * 128), &full[st]);
                ++it;
            }
        s_count[0] = it;
    } else if (warp == 1 && lane == 0) {
        // MMA issuer
        constexpr uint32_t idesc = make_idesc_tf32(128, QN);
        uint32_t it = 0, tl = 0;
        bool ok = true;
        for (int64_t t = blockIdx.x; t < tiles && ok; t += gridDim.x, ++tl) {
            const uint32_t acc = tl & 1u;
            if (!lane_wait(&tempty[acc], ((tl >> 1) & 1u) ^ 1u, abort_flag, spin)) break;
            tc_fence_after();
            for (int sl = 0; sl < nsl; ++sl) {
                const int st = int(it % STAGES);
                if (!lane_wait(&full[st], (it / STAGES) & 1u, abort_flag, spin)) { ok = false; break; }
                tc_fence_after();
                const uint32_t a0 = smem_u32(sA + st * A_TILE);
                const uint32_t b0 = smem_u32(sB + size_t(sl) * QN * 128);
#pragma unroll
                for (int k = 0; k < 4; ++k)
                    umma_tf32(tmem + acc * QN, make_desc(a0 + k * 32), make_desc(b0 + k * 32), idesc,
                              (sl > 0 || k > 0) ? 1u : 0u);
                umma_commit(&empty[st]);
                ++it;
            }
            if (ok) umma_commit(&tfull[acc]);
        }
        s_count[1] = it;
    } else if (warp >= 2) {
        // epilogue: warp w reads TMEM lanes 32 (w % 4) .. (its 32 pixels of the tile)
        const int q = warp & 3;
        uint32_t tl = 0;
        for (int64_t t = blockIdx.x; t < tiles; t += gridDim.x, ++tl) {
            const uint32_t acc = tl & 1u;
            int ok = 1;
            if (lane == 0) ok = lane_wait(&tfull[acc], (tl >> 1) & 1u, abort_flag, spin) ? 1 : 0;
            ok = __shfl_sync(0xffffffffu, ok, 0);
            if (!ok) break;
            tc_fence_after();
            const int64_t p = t * 128 + q * 32 + lane;
            const uint32_t taddr = tmem + (uint32_t(q * 32) << 16) + acc * QN;
#pragma unroll
            for (int c = 0; c < QN; c += 16) {
                float v[16];
                tmem_ld16(taddr + uint32_t(c), v);
                if (p < P) {
                    float4 *o = reinterpret_cast<float4 *>(out + p * QN + c);
                    o[0] = make_float4(v[0], v[1], v[2], v[3]);
                    o[1] = make_float4(v[4], v[5], v[6], v[7]);
                    o[2] = make_float4(v[8], v[9], v[10], v[11]);
                    o[3] = make_float4(v[12], v[13], v[14], v[15]);
                }
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&tempty[acc]);
        }
    }
    __syncthreads();
    if (*abort_flag) {
        // nothing of this CTA may still be writing shared memory or TMEM
        if (threadIdx.x == 0) atomicExch(status, int(QR_ERR_DEVICE_TIMEOUT));
        if (warp == 0 && lane == 0) {
            const uint32_t n = s_count[0];
            for (uint32_t i = n > STAGES ? n - STAGES : 0u; i < n; ++i)
                mbar_wait(&full[i % STAGES], (i / STAGES) & 1u);
        }
        if (warp == 1 && lane == 0 && s_count[1] > 0) {
            const uint32_t last = s_count[1] - 1;
            mbar_wait(&empty[last % STAGES], (last / STAGES) & 1u);
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tmem), "r"(TMEM_COLS) : "memory");
}

// ------------------------------------------------------------ fused blend + relevance
// R[p][q] = sum_c (sum_j w_pj f_{id_pj}[c]) Q[q][c] without writing the map.
// Persistent CTAs of 13 warps, one per SM; a block is 16 x 8 screen pixels
// (the 128 TMEM lanes), in 2 x 2 pixel groups.
//   * Producer warps 5-20 own two groups each.  Per block, a warp reads its
//     groups' entries once (lane m K + j = entry j of pixel m, so K <= 8),
//     merges equal ids with __match_any_sync and keeps, per group, the list of
//     distinct rows and each row's four pixel weights in shared memory.  Then,
//     128 channels at a time, it reads each distinct row once (one warp-wide
//     512-byte load), accumulates the four pixels in FP32 in entry order per
//     pixel (eight rows in flight), rounds them to BF16 and writes them into
//     a 128-byte-swizzled K-major stage (two 64-channel slices) of a ring
//     (2 stages: a deeper ring costs L1 capacity the row reads need) -- the
//     layout the fallback relevance kernel stages.
//   * Warp 4 issues kind::f16 UMMAs (BF16 x BF16, FP32 accumulation) of each
//     stage against the resident BF16 queries into one of two TMEM
//     accumulators; warps 0-3 drain the other accumulator into R.
// Each producer warp reads only its own groups' tables, so the producers
// share nothing but the ring.  Long waits back off with __nanosleep so the
// waiting warps leave issue slots to the producers.  Same bounded waits,
// abort flag and drain as the other kernels.
constexpr int FB_PRODUCERS = 16;
constexpr int FB_THREADS = (5 + FB_PRODUCERS) * 32;   // 4 epilogue warps, 1 MMA warp, producers
constexpr int FB_MAX_STAGES = 2;
constexpr int FB_GPW = 32 / FB_PRODUCERS;             // 2 x 2 groups per producer warp
constexpr int FB_ROWS = 8;                            // row loads in flight per lane
constexpr int FB_CHUNK = 128;                        // channels per stage
constexpr int FB_STAGE_BYTES = 128 * FB_CHUNK * 2;    // 32 KB (two 64-channel BF16 slices)

__device__ __forceinline__ int64_t fb_pixel(int64_t t, int r, int W, int H, int64_t P) {
    if (W <= 0) {
        const int64_t p = t * 128 + r;
        return p < P ? p : -1;
    }
    const int tiles_x = (W + 15) >> 4;
    const int tx = int(t % tiles_x), ty = int(t / tiles_x);
    const int x = tx * 16 + (r & 15), y = ty * 8 + (r >> 4);
    return (x < W && y < H) ? int64_t(y) * W + x : -1;
}

// block row (TMEM lane) of pixel m of 2 x 2 group gi (8 groups across, 4 down)
__device__ __forceinline__ int fb_row(int gi, int m) {
    return (2 * (gi >> 3) + (m >> 1)) * 16 + 2 * (gi & 7) + (m & 1);
}

// Bounded wait with backoff; false on timeout (sets the abort flag).
__device__ __forceinline__ bool lane_wait_sleep(uint64_t *bar, uint32_t parity,
                                                volatile int *abort_flag, unsigned spin) {
    if (*abort_flag) return false;
    const uint32_t a = smem_u32(bar);
    for (unsigned i = 0; i < spin / 16 + 1; ++i) {
        uint32_t done;
        asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
                     " selp.u32 %0, 1, 0, p;\n}\n"
                     : "=r"(done) : "r"(a), "r"(parity) : "memory");
        if (done) return true;
        __nanosleep(64);
    }
    *abort_flag = 1;
    return false;
}

// 4 channels of a row at channel c, widened to FP32 (the lane's share of a
// 128-channel chunk)
template <int DT>
__device__ __forceinline__ float4 fb_load4(const unsigned char *__restrict__ feat, size_t row_bytes,
                                           int id, int c) {
    const unsigned char *ptr = feat + size_t(id) * row_bytes;
    if (DT == QR_F32) {
        return __ldg(reinterpret_cast<const float4 *>(ptr + size_t(c) * 4));
    } else if (DT == QR_BF16) {
        const uint2 u = __ldg(reinterpret_cast<const uint2 *>(ptr + size_t(c) * 2));
        return make_float4(__uint_as_float(u.x << 16), __uint_as_float(u.x & 0xFFFF0000u),
                           __uint_as_float(u.y << 16), __uint_as_float(u.y & 0xFFFF0000u));
    } else {
        const uint32_t u = __ldg(reinterpret_cast<const uint32_t *>(ptr + size_t(c)));
        const __half2_raw lo = __nv_cvt_fp8x2_to_halfraw2(__nv_fp8x2_storage_t(u & 0xFFFFu), __NV_E4M3);
        const __half2_raw hi = __nv_cvt_fp8x2_to_halfraw2(__nv_fp8x2_storage_t(u >> 16), __NV_E4M3);
        const float2 a = __half22float2(*reinterpret_cast<const __half2 *>(&lo));
        const float2 b = __half22float2(*reinterpret_cast<const __half2 *>(&hi));
        return make_float4(a.x, a.y, b.x, b.y);
    }
}

template <int DT, int QN>
__global__ void __launch_bounds__(FB_THREADS, 1)
blend_relevance_kernel(const unsigned char *__restrict__ feat, const float *__restrict__ fscale,
                       int64_t n_gauss, int C, const int32_t *__restrict__ ids,
                       const float *__restrict__ wts, const uint8_t *__restrict__ cnt, int64_t P,
                       int K, int W, int H, const uint16_t *__restrict__ queries,
                       float *__restrict__ out, int *__restrict__ status, int FB_STAGES,
                       unsigned spin) {
    constexpr uint32_t TMEM_COLS = 2 * QN < 32 ? 32 : 2 * QN;
    constexpr int ESZ = DT == QR_F32 ? 4 : DT == QR_BF16 ? 2 : 1;
    constexpr unsigned FULL = 0xffffffffu;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char *base = reinterpret_cast<unsigned char *>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    const int nchunk = C / FB_CHUNK;
    const int nslices = C / BK;                                      // 64-channel query slices
    unsigned char *sA = base;                                        // FB_STAGES x 32 KB
    unsigned char *sB = sA + FB_STAGES * FB_STAGE_BYTES;             // nslices x QN x 128 B
    int32_t *t_id = reinterpret_cast<int32_t *>(sB + size_t(nslices) * QN * 128);   // [32 groups][32]
    float4 *t_w = reinterpret_cast<float4 *>(t_id + 32 * 32);                         // [32][32] weights of the 4 pixels
    int32_t *t_n = reinterpret_cast<int32_t *>(t_w + 32 * 32);                        // [32] distinct rows per group
    uint64_t *full = reinterpret_cast<uint64_t *>(t_n + 32);
    uint64_t *empty = full + FB_MAX_STAGES;
    uint64_t *tfull = empty + FB_MAX_STAGES;
    uint64_t *tempty = tfull + 2;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(tempty + 2);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);
    uint32_t *s_count = reinterpret_cast<uint32_t *>(tmem_slot + 2);   // [0] MMA stages issued
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    // queries -> swizzled K-major BF16 slices of 64 channels (16-byte chunks copied as they are)
    for (int i = threadIdx.x; i < nslices * QN * 8; i += FB_THREADS) {
        const int sl = i / (QN * 8), rem = i % (QN * 8), n = rem >> 3, c = rem & 7;
        const uint4 v = *reinterpret_cast<const uint4 *>(queries + size_t(n) * C + sl * BK + c * 8);
        *reinterpret_cast<uint4 *>(sB + size_t(sl) * QN * 128 + swz(n, c)) = v;
    }
    if (threadIdx.x == 0) {
        for (int st = 0; st < FB_STAGES; ++st) {
            mbar_init(&full[st], FB_PRODUCERS);
            mbar_init(&empty[st], 1);
        }
        for (int a = 0; a < 2; ++a) {
            mbar_init(&tfull[a], 1);
            mbar_init(&tempty[a], 4);
        }
        *abort_flag = 0;
        s_count[0] = 0u;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 4) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     :: "r"(smem_u32(tmem_slot)), "r"(TMEM_COLS) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    const int64_t tiles = (W > 0) ? int64_t((W + 15) >> 4) * ((H + 7) >> 3) : (P + 127) / 128;
    const size_t row_bytes = size_t(C) * ESZ;

    if (warp >= 5) {
        const int pw = warp - 5;
        const int m = lane / K, j = lane - m * K;      // entry j of group pixel m (m < 4)
        uint32_t it = 0;
        bool ok = true;
        for (int64_t t = blockIdx.x; t < tiles; t += gridDim.x) {
            // the distinct rows of this warp's groups and their pixel weights
#pragma unroll
            for (int q4 = 0; q4 < FB_GPW; ++q4) {
                if (!ok) break;
                const int gi = pw + FB_PRODUCERS * q4;
                int id = -1;
                float w = 0.f;
                if (m < 4) {
                    const int64_t p = fb_pixel(t, fb_row(gi, m), W, H, P);
                    if (p >= 0 && j < int(cnt[p])) {
                        id = ids[p * K + j];
                        w = wts[p * K + j];
                        if (uint64_t(int64_t(id)) >= uint64_t(n_gauss)) { id = -1; w = 0.f; }
                        else if (DT == QR_FP8E4M3) w *= fscale[id];
                    }
                }
                const unsigned peers = __match_any_sync(FULL, id);
                const int leader = __ffs(peers) - 1;
                const unsigned leaders = __ballot_sync(FULL, id >= 0 && lane == leader);
                const int slot = __popc(leaders & ((1u << leader) - 1u));
                float4 *tw = t_w + gi * 32;
                tw[lane] = make_float4(0.f, 0.f, 0.f, 0.f);
                __syncwarp();
                if (id >= 0) {
                    // a pixel listing an id twice gets the sum of its weights
                    float *wrow = reinterpret_cast<float *>(&tw[slot]);
                    atomicAdd(wrow + m, w);
                    if (lane == leader) t_id[gi * 32 + slot] = id;
                }
                if (lane == 0) t_n[gi] = __popc(leaders);
                __syncwarp();
            }
            for (int ch = 0; ch < nchunk && ok; ++ch) {
                const int st = int(it % FB_STAGES);
                int wok = 1;
                if (lane == 0) wok = lane_wait_sleep(&empty[st], ((it / FB_STAGES) & 1u) ^ 1u, abort_flag, spin) ? 1 : 0;
                wok = __shfl_sync(FULL, wok, 0);
                if (!wok) { ok = false; break; }
                unsigned char *stage = sA + st * FB_STAGE_BYTES;
                const int c = ch * FB_CHUNK + lane * 4;
                for (int q4 = 0; q4 < FB_GPW; ++q4) {
                    const int gi = pw + FB_PRODUCERS * q4;
                    const int nr = t_n[gi];
                    const int32_t *tid = t_id + gi * 32;
                    const float4 *tw = t_w + gi * 32;
                    float4 acc[4];
#pragma unroll
                    for (int mm = 0; mm < 4; ++mm) acc[mm] = make_float4(0.f, 0.f, 0.f, 0.f);
                    for (int r0 = 0; r0 < nr; r0 += FB_ROWS) {
                        float4 f[FB_ROWS];
#pragma unroll
                        for (int u = 0; u < FB_ROWS; ++u)
                            f[u] = r0 + u < nr ? fb_load4<DT>(feat, row_bytes, tid[r0 + u], c)
                                               : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
                        for (int u = 0; u < FB_ROWS; ++u) {
                            if (r0 + u >= nr) break;
                            const float4 wg = tw[r0 + u];
                            const float wv[4] = {wg.x, wg.y, wg.z, wg.w};
#pragma unroll
                            for (int mm = 0; mm < 4; ++mm) {
                                acc[mm].x = fmaf(wv[mm], f[u].x, acc[mm].x);
                                acc[mm].y = fmaf(wv[mm], f[u].y, acc[mm].y);
                                acc[mm].z = fmaf(wv[mm], f[u].z, acc[mm].z);
                                acc[mm].w = fmaf(wv[mm], f[u].w, acc[mm].w);
                            }
                        }
                    }
                    // BF16 into the stage: channel 4 lane of the chunk lies in
                    // 64-channel slice lane / 16, 16-byte chunk (lane % 16) / 2
#pragma unroll
                    for (int mm = 0; mm < 4; ++mm) {
                        const int r = fb_row(gi, mm);
                        const __nv_bfloat162 lo = __floats2bfloat162_rn(acc[mm].x, acc[mm].y);
                        const __nv_bfloat162 hi = __floats2bfloat162_rn(acc[mm].z, acc[mm].w);
                        uint2 packed;
                        packed.x = *reinterpret_cast<const uint32_t *>(&lo);
                        packed.y = *reinterpret_cast<const uint32_t *>(&hi);
                        *reinterpret_cast<uint2 *>(stage + (lane >> 4) * (128 * 128) +
                                                   swz(r, (lane & 15) >> 1) + (lane & 1) * 8) = packed;
                    }
                }
                fence_async_smem();
                __syncwarp();
                if (lane == 0) mbar_arrive(&full[st]);
                ++it;
            }
        }
    } else if (warp == 4 && lane == 0) {
        // MMA issuer: per stage two 64-channel slices, four K = 16 steps each
        constexpr uint32_t idesc = make_idesc(128, QN);
        uint32_t it = 0, tl = 0;
        bool ok = true;
        for (int64_t t = blockIdx.x; t < tiles && ok; t += gridDim.x, ++tl) {
            const uint32_t acc = tl & 1u;
            if (!lane_wait_sleep(&tempty[acc], ((tl >> 1) & 1u) ^ 1u, abort_flag, spin)) break;
            tc_fence_after();
            for (int ch = 0; ch < nchunk; ++ch) {
                const int st = int(it % FB_STAGES);
                if (!lane_wait_sleep(&full[st], (it / FB_STAGES) & 1u, abort_flag, spin)) { ok = false; break; }
                tc_fence_after();
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const uint32_t a0 = smem_u32(sA + st * FB_STAGE_BYTES + h * (128 * 128));
                    const uint32_t b0 = smem_u32(sB + size_t(2 * ch + h) * QN * 128);
#pragma unroll
                    for (int k = 0; k < BK / 16; ++k)
                        umma_bf16(tmem + acc * QN, make_desc(a0 + k * 32), make_desc(b0 + k * 32),
                                  idesc, (ch > 0 || h > 0 || k > 0) ? 1u : 0u);
                }
                umma_commit(&empty[st]);
                ++it;
            }
            if (ok) umma_commit(&tfull[acc]);
        }
        s_count[0] = it;
    } else if (warp < 4) {
        // epilogue: warp q reads TMEM lanes 32 q .. (block rows 32 q .. 32 q + 31)
        const int q = warp;
        uint32_t tl = 0;
        for (int64_t t = blockIdx.x; t < tiles; t += gridDim.x, ++tl) {
            const uint32_t acc = tl & 1u;
            int ok = 1;
            if (lane == 0) ok = lane_wait_sleep(&tfull[acc], (tl >> 1) & 1u, abort_flag, spin) ? 1 : 0;
            ok = __shfl_sync(FULL, ok, 0);
            if (!ok) break;
            tc_fence_after();
            const int64_t p = fb_pixel(t, q * 32 + lane, W, H, P);
            const uint32_t taddr = tmem + (uint32_t(q * 32) << 16) + acc * QN;
#pragma unroll
            for (int c = 0; c < QN; c += 16) {
                float v[16];
                tmem_ld16(taddr + uint32_t(c), v);
                if (p >= 0) {
                    float4 *o = reinterpret_cast<float4 *>(out + p * QN + c);
                    o[0] = make_float4(v[0], v[1], v[2], v[3]);
                    o[1] = make_float4(v[4], v[5], v[6], v[7]);
                    o[2] = make_float4(v[8], v[9], v[10], v[11]);
                    o[3] = make_float4(v[12], v[13], v[14], v[15]);
                }
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&tempty[acc]);
        }
    }
    __syncthreads();
    if (*abort_flag) {
        if (threadIdx.x == 0) atomicExch(status, int(QR_ERR_DEVICE_TIMEOUT));
        // the MMAs of the last issued stage must have finished reading shared memory
        if (warp == 4 && lane == 0 && s_count[0] > 0) {
            const uint32_t last = s_count[0] - 1;
            mbar_wait(&empty[last % FB_STAGES], (last / FB_STAGES) & 1u);
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 4)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tmem), "r"(TMEM_COLS) : "memory");
}

size_t fb_smem_with(int stages, int Q, int C) {
    return 1024 + size_t(stages) * FB_STAGE_BYTES + size_t(C / BK) * Q * 128 +
           size_t(32) * 32 * (4 + 16) + 32 * 4 + 256;
}
// the deepest ring (4, 3 or 2 stages) that fits next to the queries
int fb_stages(int Q, int C) {
    for (int st = FB_MAX_STAGES; st >= 2; --st)
        if (fb_smem_with(st, Q, C) <= 227 * 1024) return st;
    return 0;
}
size_t fb_smem_bytes(int Q, int C, int) {
    const int st = fb_stages(Q, C);
    return st ? fb_smem_with(st, Q, C) : ~size_t(0);
}

template <int DT, int QN>
cudaError_t run_fused(const void *feat, const float *scale, int64_t n_gauss, int C,
                      const int32_t *ids, const float *w, const uint8_t *cnt, int64_t P, int K,
                      int W, int H, const uint16_t *q, float *out, int *status, cudaStream_t s) {
    const size_t smem = fb_smem_bytes(QN, C, K);
    cudaError_t e = cudaFuncSetAttribute(blend_relevance_kernel<DT, QN>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t tiles = (W > 0) ? int64_t((W + 15) >> 4) * ((H + 7) >> 3) : (P + 127) / 128;
    const int grid = int(tiles < sms ? tiles : sms);
    blend_relevance_kernel<DT, QN><<<grid, FB_THREADS, smem, s>>>(
        static_cast<const unsigned char *>(feat), scale, n_gauss, C, ids, w, cnt, P, K, W, H, q,
        out, status, fb_stages(QN, C), g_wait_limit);
    count_launch();
    return cudaGetLastError();
}

template <int DT>
cudaError_t fused_q(const void *feat, const float *scale, int64_t n_gauss, int C, const int32_t *ids,
                    const float *w, const uint8_t *cnt, int64_t P, int K, int W, int H,
                    const uint16_t *q, int Q, float *out, int *status, cudaStream_t s) {
    switch (Q) {
        case 16: return run_fused<DT, 16>(feat, scale, n_gauss, C, ids, w, cnt, P, K, W, H, q, out, status, s);
        case 32: return run_fused<DT, 32>(feat, scale, n_gauss, C, ids, w, cnt, P, K, W, H, q, out, status, s);
        case 64: return run_fused<DT, 64>(feat, scale, n_gauss, C, ids, w, cnt, P, K, W, H, q, out, status, s);
        case 128: return run_fused<DT, 128>(feat, scale, n_gauss, C, ids, w, cnt, P, K, W, H, q, out, status, s);
    }
    return cudaErrorInvalidValue;
}

size_t tma_smem_bytes(int Q, int C) {
    return 1024 + size_t(STAGES) * A_TILE + size_t(C) * Q * 4 + 256;
}

template <int QN>
cudaError_t run_tma(const float *map, const uint16_t *q, int64_t P, int C, float *out, int *status,
                    cudaStream_t s) {
    EncodeTiled enc = tensor_map_encoder();
    if (!enc) return cudaErrorNotSupported;
    CUtensorMap tm;
    const cuuint64_t dims[2] = {cuuint64_t(C), cuuint64_t(P)};
    const cuuint64_t strides[1] = {cuuint64_t(C) * 4};
    const cuuint32_t box[2] = {32, 128};
    const cuuint32_t estr[2] = {1, 1};
    if (enc(&tm, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float *>(map), dims, strides, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return cudaErrorInvalidValue;
    const size_t smem = tma_smem_bytes(QN, C);
    cudaError_t e = cudaFuncSetAttribute(relevance_tma_kernel<QN>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t tiles = (P + 127) / 128;
    const int grid = int(tiles < sms ? tiles : sms);
    relevance_tma_kernel<QN><<<grid, TT, smem, s>>>(tm, q, P, C, out, status, g_wait_limit);
    count_launch();
    return cudaGetLastError();
}

template <int QN>
cudaError_t run(const float *map, const uint16_t *q, int64_t P, int C, float *out, int *status,
                cudaStream_t s) {
    const size_t smem = 1024 + size_t(C / BK) * QN * 128 + 2 * A_STAGE + 64;
    cudaError_t e = cudaFuncSetAttribute(relevance_kernel<QN>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         int(smem));
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t tiles = (P + BM - 1) / BM;
    const int64_t cap = int64_t(sms) * 2;      // two resident CTAs per SM
    const int grid = int(tiles < cap ? tiles : cap);
    relevance_kernel<QN><<<grid, NT, smem, s>>>(map, q, P, C, out, status);
    count_launch();
    return cudaGetLastError();
}

}  // namespace

void set_wait_limit(unsigned polls) { g_wait_limit = polls ? polls : kSpinLimit; }

bool blend_relevance_supported(qr_dtype dt, int Q, int C, int K) {
    if (C < FB_CHUNK || C % FB_CHUNK || K < 1 || K > 8) return false;
    if (!(Q == 16 || Q == 32 || Q == 64 || Q == 128)) return false;
    (void)dt;
    return fb_smem_bytes(Q, C, K) <= 227 * 1024;
}

cudaError_t launch_blend_relevance(const void *feat, const float *scale, qr_dtype dt, int C,
                                   int64_t n_gauss, const int32_t *ids, const float *w,
                                   const uint8_t *cnt, int64_t P, int K, int W, int H,
                                   const uint16_t *q, int Q, float *out, int *status,
                                   cudaStream_t s) {
    switch (dt) {
        case QR_F32: return fused_q<QR_F32>(feat, scale, n_gauss, C, ids, w, cnt, P, K, W, H, q, Q, out, status, s);
        case QR_BF16: return fused_q<QR_BF16>(feat, scale, n_gauss, C, ids, w, cnt, P, K, W, H, q, Q, out, status, s);
        case QR_FP8E4M3: return fused_q<QR_FP8E4M3>(feat, scale, n_gauss, C, ids, w, cnt, P, K, W, H, q, Q, out, status, s);
    }
    return cudaErrorInvalidValue;
}

bool relevance_supported(int Q, int C) {
    if (C < BK || C % BK) return false;
    if (!(Q == 16 || Q == 32 || Q == 64 || Q == 128)) return false;
    return 1024 + size_t(C / BK) * Q * 128 + 2 * A_STAGE + 64 <= 227 * 1024;
}

// The TMA + TF32 kernel where its shared memory fits (the queries are held in
// FP32), else the register-staged BF16 kernel.
static bool tma_fits(int Q, int C, int64_t P, const float *map) {
    return C % 32 == 0 && P < (int64_t(1) << 31) - 128 &&
           (reinterpret_cast<uintptr_t>(map) & 15) == 0 && tma_smem_bytes(Q, C) <= 227 * 1024;
}

cudaError_t launch_relevance(const float *map, const uint16_t *q, int Q, int64_t P, int C,
                             float *out, int *status, cudaStream_t s) {
    if (tma_fits(Q, C, P, map)) {
        switch (Q) {
            case 16: return run_tma<16>(map, q, P, C, out, status, s);
            case 32: return run_tma<32>(map, q, P, C, out, status, s);
            case 64: return run_tma<64>(map, q, P, C, out, status, s);
            case 128: return run_tma<128>(map, q, P, C, out, status, s);
        }
    }
    switch (Q) {
        case 16: return run<16>(map, q, P, C, out, status, s);
        case 32: return run<32>(map, q, P, C, out, status, s);
        case 64: return run<64>(map, q, P, C, out, status, s);
        case 128: return run<128>(map, q, P, C, out, status, s);
    }
    return cudaErrorInvalidValue;
}

}  // namespace qr
