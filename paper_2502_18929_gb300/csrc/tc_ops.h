// bf16 tensor-core helpers shared by the learned proposal's inference
// (kernels.cu) and training (learn.cu) kernels.
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace qmc {

// Two floats as one bf16x2 word (rounded to nearest even); lo in the low half
// (the lower column of a fragment pair).
__device__ __forceinline__ uint32_t bf16x2(float lo, float hi)
{
    const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<const uint32_t*>(&v);
}

// D += A B for one m16n8k16 tile: A 16x16 bf16 (row-major fragment a[4]),
// B 16x8 bf16 (column fragment b0, b1), D 16x8 fp32.  Fragment ownership
// (g = lane / 4, q = lane % 4): a0 (row g, cols 2q, 2q+1), a1 (row g+8),
// a2 (row g, cols 2q+8, 2q+9), a3 (row g+8, cols 2q+8, 2q+9); b0 (rows 2q,
// 2q+1, col g), b1 (rows 2q+8, 2q+9, col g); d0 d1 (row g, cols 2q, 2q+1),
// d2 d3 (row g+8).
__device__ __forceinline__ void mma_bf16(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1)
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// tanh(x) by the hardware approximation (tanh.approx.f32).
__device__ __forceinline__ float tanh_fast(float x)
{
    float y;
    asm("tanh.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// GELU in its tanh form, 0.5 x (1 + tanh(sqrt(2/pi) (x + 0.044715 x^3))),
// every product and sum rounded as written.
__device__ __forceinline__ float tc_gelu(float x)
{
    const float u = __fmul_rn(0.7978845608028654f, __fadd_rn(x, __fmul_rn(0.044715f, __fmul_rn(x, __fmul_rn(x, x)))));
    return __fmul_rn(__fmul_rn(0.5f, x), __fadd_rn(1.0f, tanh_fast(u)));
}

// d GELU / dx of the tanh form: 0.5 (1 + tanh u) + 0.5 x (1 - tanh^2 u) du/dx,
// du/dx = sqrt(2/pi) (1 + 3 * 0.044715 x^2).
__device__ __forceinline__ float tc_gelu_prime(float x)
{
    const float u = 0.7978845608028654f * (x + 0.044715f * x * x * x);
    const float th = tanh_fast(u);
    return 0.5f * (1.0f + th) + 0.5f * x * (1.0f - th * th) * 0.7978845608028654f * (1.0f + 0.134145f * x * x);
}

} // namespace qmc
