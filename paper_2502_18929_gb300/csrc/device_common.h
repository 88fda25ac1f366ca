// Device helpers shared by the step kernels of both key widths: Philox, the
// walker draws' counters, the sticky error flag, segment lookup.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "kernels.h"
#include "qmc_types.h"

namespace qmc {

constexpr uint32_t kFull = 0xFFFFFFFFu;

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon et al., SC'11).
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint4 philox10(uint4 c, uint2 k)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
        c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
        k.x += 0x9E3779B9u;
        k.y += 0xBB67AE85u;
    }
    return c;
}

__device__ __forceinline__ int64_t iabs64(int64_t v) { return v < 0 ? -v : v; }

__device__ __forceinline__ void set_error(DevState* st, uint32_t code)
{
    atomicCAS(&st->error, 0u, code);
}

__device__ __forceinline__ uint32_t read_error(const DevState* st)
{
    return *(volatile const uint32_t*)&st->error;
}

// The error flag as one CTA sees it: read once and shared, so that every
// thread of the CTA takes the same early exit (another CTA may raise the flag
// while this one starts).
__device__ __forceinline__ bool cta_error(const DevState* st)
{
    __shared__ uint32_t s_err;
    if (threadIdx.x == 0) s_err = read_error(st);
    __syncthreads();
    return s_err != 0;
}

// Segment of record i in a population slot: upper_bound(off[1..nseg], i).
__device__ __forceinline__ int seg_of(const int64_t* off, int nseg, int64_t i)
{
    int lo = 0, hi = nseg - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (__ldg(&off[mid]) <= i) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// The walker draw's counters [reading R3]: for the parent at rank r of its
// vector (index in the key-sorted population) in pass phase, walker w (real
// walkers first) has T = W << 20 | L with W word r % 4 of the rank group's
// call of level w (w = 0, 1) or word (w - 2) % 4 of the parent's call
// (w - 2) / 4 (w >= 2), and L the top 20 bits of word 0 of the walker's own
// call (component comp, index j).
__device__ __forceinline__ uint4 group_words(uint32_t g, uint32_t level, int phase, uint2 kd)
{
    return philox10(make_uint4(g, level, (uint32_t)phase | (kKindGroup << 2), 0u), kd);
}

__device__ __forceinline__ uint4 extra_words(uint32_t rank, uint32_t b, int phase, uint2 kd)
{
    return philox10(make_uint4(rank, b, (uint32_t)phase | (kKindExtra << 2), 0u), kd);
}

__device__ __forceinline__ int64_t walker_T(uint32_t W, uint32_t rank, uint32_t j, int comp, int phase, uint2 kd)
{
    const uint4 o = philox10(make_uint4(rank, j, (uint32_t)phase | ((uint32_t)comp << 1) | (kKindLow << 2), 0u), kd);
    return (int64_t)((((uint64_t)W) << 20) | (o.x >> 12));
}

__device__ __forceinline__ uint32_t word_of(const uint4& o, int k)
{
    return k == 0 ? o.x : (k == 1 ? o.y : (k == 2 ? o.z : o.w));
}

} // namespace qmc
