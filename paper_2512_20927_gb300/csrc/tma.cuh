// TMA (cp.async.bulk.tensor) and mbarrier helpers shared by the kernels that
// stage tiles with the tensor memory accelerator, and the host-side tensor-map
// encoder (the driver's cuTensorMapEncodeTiled, resolved once through the
// runtime, so the library does not link against libcuda).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>

namespace qr {

__device__ __forceinline__ uint32_t tma_smem_addr(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void tma_mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(tma_smem_addr(bar)), "r"(count)
                 : "memory");
}

// Make initialised barriers visible to the TMA unit.
__device__ __forceinline__ void tma_fence_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// Bounded wait for the phase with the given parity; false after `limit` polls.
__device__ __forceinline__ bool tma_mbar_wait(uint64_t *bar, uint32_t parity, unsigned limit) {
    const uint32_t a = tma_smem_addr(bar);
    for (unsigned i = 0; i < limit; ++i) {
        uint32_t done;
        asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
                     " selp.u32 %0, 1, 0, p;\n}\n"
                     : "=r"(done) : "r"(a), "r"(parity) : "memory");
        if (done) return true;
    }
    return false;
}

// Arrive on the barrier announcing the bytes the next TMA copy delivers.
__device__ __forceinline__ void tma_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;"
                 :: "r"(tma_smem_addr(bar)), "r"(bytes) : "memory");
}

// 3-D tiled TMA load of the map's box at (x, y, z) (x innermost; x * element
// size must be a multiple of 16 bytes) into shared memory; completion counted
// on bar.  Out-of-range elements are filled with zeros.
__device__ __forceinline__ void tma_load_3d(void *dst, const CUtensorMap *map, int x, int y, int z,
                                            uint64_t *bar) {
    asm volatile("cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
                 " [%0], [%1, {%2, %3, %4}], [%5];"
                 :: "r"(tma_smem_addr(dst)), "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y),
                    "r"(z), "r"(tma_smem_addr(bar)) : "memory");
}

using EncodeTiled = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *,
                                 const cuuint64_t *, const cuuint64_t *, const cuuint32_t *,
                                 const cuuint32_t *, CUtensorMapInterleave, CUtensorMapSwizzle,
                                 CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

// The driver's tensor-map encoder, or nullptr if the driver has none.
inline EncodeTiled tensor_map_encoder() {
    static std::once_flag once;
    static EncodeTiled fn = nullptr;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess && q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiled>(p);
    });
    return fn;
}

}  // namespace qr
