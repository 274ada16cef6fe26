// Tensor-core products with FP32-class accuracy from TF32 operands
// (mma.sync m16n8k8, FP32 accumulation), shared by the Eq. 2 kernel and the
// backward's per-tile partial rows.  Each FP32 operand is split as
// x = hi + lo with hi, lo TF32 (round to nearest) and a step takes the three
// products lo*hi + hi*lo + hi*hi: the dropped lo*lo term and the rounding of
// lo leave about 2^-22 of |x||y| per product.
//
// Fragments of m16n8k8 (g = lane / 4, t = lane % 4):
//   A (16 x 8, row-major): a0 = A[g][t], a1 = A[g + 8][t], a2 = A[g][t + 4], a3 = A[g + 8][t + 4];
//   B (8 x 8):             b0 = B[t][g], b1 = B[t + 4][g];
//   C / D (16 x 8):        c0 = D[g][2t], c1 = D[g][2t + 1], c2 = D[g + 8][2t], c3 = D[g + 8][2t + 1].
#pragma once

#include <stdint.h>

namespace qr {

__device__ __forceinline__ uint32_t to_tf32(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ void split_tf32(float x, uint32_t &hi, uint32_t &lo) {
    hi = to_tf32(x);
    lo = to_tf32(x - __uint_as_float(hi));
}
__device__ __forceinline__ void mma_tf32(float (&d)[4], uint32_t a0, uint32_t a1, uint32_t a2,
                                         uint32_t a3, uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
        "{%8,%9}, {%0,%1,%2,%3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}
// d += A B with A = ah + al, B = bh + bl (the small products first)
__device__ __forceinline__ void mma3(float (&d)[4], const uint32_t (&ah)[4], const uint32_t (&al)[4],
                                     uint32_t bh0, uint32_t bh1, uint32_t bl0, uint32_t bl1) {
    mma_tf32(d, al[0], al[1], al[2], al[3], bh0, bh1);
    mma_tf32(d, ah[0], ah[1], ah[2], ah[3], bl0, bl1);
    mma_tf32(d, ah[0], ah[1], ah[2], ah[3], bh0, bh1);
}

}  // namespace qr
