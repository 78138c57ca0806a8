// mma_tf32.cuh -- FP32 products on the tensor cores as 3xTF32: x = hi + lo,
// hi = tf32(x), lo = tf32(x - hi); a b ~ hi_a hi_b + hi_a lo_b + lo_a hi_b,
// each term an mma.sync.m16n8k8 with FP32 accumulation.  Fragment layout of
// m16n8k8 (g = lane / 4, c = lane % 4): A a0..a3 = (g, c), (g+8, c), (g, c+4),
// (g+8, c+4); B b0, b1 = (k=c, n=g), (k=c+4, n=g); D d0..d3 = (g, 2c),
// (g, 2c+1), (g+8, 2c), (g+8, 2c+1).
#pragma once

#include <cstdint>

namespace dmrg {

__device__ __forceinline__ void split_tf32(float x, uint32_t &hi, uint32_t &lo)
{
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(hi) : "f"(x));
    const float r = x - __uint_as_float(hi);
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(lo) : "f"(r));
}

__device__ __forceinline__ void mma_tf32(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1)
{
    asm volatile("mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
                 "{%0,%1,%2,%3};"
                 : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
                 : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// 3xTF32 product into d: A rows/columns from `arow(r, k)`, B from `bcol(k, n)`
template <typename FA, typename FB>
__device__ __forceinline__ void mma3(float (&d)[4], int g, int c, FA arow, FB bcol, int m0, int n0, int k0)
{
    uint32_t ah[4], al[4], bh0, bl0, bh1, bl1;
    split_tf32(arow(m0 + g, k0 + c), ah[0], al[0]);
    split_tf32(arow(m0 + g + 8, k0 + c), ah[1], al[1]);
    split_tf32(arow(m0 + g, k0 + c + 4), ah[2], al[2]);
    split_tf32(arow(m0 + g + 8, k0 + c + 4), ah[3], al[3]);
    split_tf32(bcol(k0 + c, n0 + g), bh0, bl0);
    split_tf32(bcol(k0 + c + 4, n0 + g), bh1, bl1);
    mma_tf32(d, al, bh0, bh1);
    mma_tf32(d, ah, bl0, bl1);
    mma_tf32(d, ah, bh0, bh1);
}

}  // namespace dmrg
