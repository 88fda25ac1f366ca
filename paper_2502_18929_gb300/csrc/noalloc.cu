// Per-vector observables of caller-owned device populations without any
// device allocation (qmc_observables_noalloc in include/qmc.h).
//
// The accumulators live in a file-scope static device array; every GPU that
// loads the library holds it until the process exits.  Host code cannot use
// the array's name as a device address, so the address is looked up once per
// device with cudaGetSymbolAddress (with that device current) and cached.
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>

#include "../../include/qmc.h"

namespace {

struct ObsAcc {
    unsigned long long count;
    long long ntot, dre, dim;
};

static __device__ __align__(256) ObsAcc g_noalloc_acc[QMC_NOALLOC_MAX_SEGMENTS];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
ObsAcc* g_acc_ptr[kMaxDevices] = {};

__global__ void k_noalloc_clear(ObsAcc* acc, int nseg)
{
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < nseg; s += gridDim.x * blockDim.x)
        acc[s] = ObsAcc{0ull, 0ll, 0ll, 0ll};
}

__device__ __forceinline__ int seg_index(const int64_t* off, int nseg, int64_t i)
{
    int lo = 0, hi = nseg - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (off[mid] <= i) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// Add the warp's per-lane sums to the accumulators, one set of atomics per
// vector the warp holds.  Lanes hold nondecreasing vector indices (each lane
// walks consecutive records of the warp's range), so the lanes of one vector
// are contiguous: a segmented sum down the warp leaves each vector's total in
// its first lane.  seg < 0: the lane holds nothing.
__device__ __forceinline__ void warp_flush(ObsAcc* acc, int seg, unsigned long long cnt, long long ntot,
                                           long long dre, long long dim, int lane)
{
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const int so = __shfl_down_sync(0xFFFFFFFFu, seg, d);
        const unsigned long long c = __shfl_down_sync(0xFFFFFFFFu, cnt, d);
        const long long t = __shfl_down_sync(0xFFFFFFFFu, ntot, d);
        const long long r = __shfl_down_sync(0xFFFFFFFFu, dre, d);
        const long long i = __shfl_down_sync(0xFFFFFFFFu, dim, d);
        if (lane + d < 32 && so == seg) {
            cnt += c;
            ntot += t;
            dre += r;
            dim += i;
        }
    }
    const int up = __shfl_up_sync(0xFFFFFFFFu, seg, 1);
    if (seg >= 0 && (lane == 0 || up != seg) && cnt) {
        atomicAdd(&acc[seg].count, cnt);
        atomicAdd((unsigned long long*)&acc[seg].ntot, (unsigned long long)ntot);
        if (dre) atomicAdd((unsigned long long*)&acc[seg].dre, (unsigned long long)dre);
        if (dim) atomicAdd((unsigned long long*)&acc[seg].dim, (unsigned long long)dim);
    }
}

// records: 16-byte (uint64 key, int32 re, int32 im), keys (x << n) | y;
// vector s holds records [off[s], off[s + 1]).  Each warp owns a contiguous
// range of [off[0], off[nseg]); lane l takes its records l, l + 32, ...
// and sums them per vector in registers, so a vector costs one set of
// atomics per warp that touches it instead of one per record.
__global__ void k_noalloc_accumulate(const uint4* __restrict__ rec, const int64_t* __restrict__ off, int nseg, int n,
                                     ObsAcc* acc)
{
    const int lane = threadIdx.x & 31;
    const int64_t first = off[0], total = off[nseg] - first;
    const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x >> 5);
    const int64_t gw = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int64_t chunk = ((total + nwarps - 1) / nwarps + 31) / 32 * 32;
    const int64_t wb = first + min(total, gw * chunk), we = first + min(total, (gw + 1) * chunk);
    const uint32_t ymask = n == 32 ? 0xFFFFFFFFu : ((1u << n) - 1u);
    int cur = -1;
    int64_t cur_end = -1;
    unsigned long long cnt = 0ull;
    long long ntot = 0, dre = 0, dim = 0;
    for (int64_t j = wb; j < we; j += 32) {
        const int64_t i = j + lane;
        const bool valid = i < we;
        int s = valid ? cur : -1;   // a lane past the range holds nothing (keeps lanes' vectors nondecreasing)
        if (valid && i >= cur_end) {
            s = seg_index(off, nseg, i);
            cur_end = off[s + 1];
        }
        if (__any_sync(0xFFFFFFFFu, s != cur)) {
            warp_flush(acc, cur, cnt, ntot, dre, dim, lane);
            cur = s;
            cnt = 0ull;
            ntot = dre = dim = 0;
        }
        if (valid) {
            const uint4 r = __ldcs(rec + i);
            const uint64_t key = ((uint64_t)r.y << 32) | r.x;
            const int32_t re = (int32_t)r.z, im = (int32_t)r.w;
            cnt += 1ull;
            ntot += (re < 0 ? -(long long)re : re) + (im < 0 ? -(long long)im : im);
            if ((uint32_t)(key >> n) == (uint32_t)(key & ymask)) {
                dre += re;
                dim += im;
            }
        }
    }
    warp_flush(acc, cur, cnt, ntot, dre, dim, lane);
}

__global__ void k_noalloc_store(const ObsAcc* acc, int nseg, qmc_obs* out)
{
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < nseg; s += gridDim.x * blockDim.x)
        out[s] = qmc_obs{(int64_t)acc[s].count, acc[s].ntot, acc[s].dre, acc[s].dim};
}

// Device address of the accumulator array on the current device (set-up on
// the first call per device).
int acc_address(ObsAcc** out)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return QMC_ERR_CUDA;
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_acc_ptr[dev]) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_acc);
        if (e != cudaSuccess || p == nullptr) {
            cudaGetLastError();
            return QMC_ERR_CUDA;
        }
        g_acc_ptr[dev] = (ObsAcc*)p;
    }
    *out = g_acc_ptr[dev];
    return QMC_OK;
}

} // namespace

extern "C" int qmc_observables_noalloc(const void* records, const int64_t* seg_offsets, int32_t n_segments,
                                       int32_t n_qubits, qmc_obs* out, void* cuda_stream)
{
    if (!records || !seg_offsets || !out || n_segments < 1 || n_qubits < 1 || n_qubits > 32)
        return QMC_ERR_INVALID_ARG;
    if (n_segments > QMC_NOALLOC_MAX_SEGMENTS) return QMC_ERR_INVALID_ARG;
    if (((uintptr_t)records & 15u) != 0 || ((uintptr_t)seg_offsets & 7u) != 0) return QMC_ERR_INVALID_ARG;
    ObsAcc* acc = nullptr;
    int rc = acc_address(&acc);
    if (rc != QMC_OK) return rc;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    const int blocks_seg = (n_segments + 255) / 256;
    k_noalloc_clear<<<blocks_seg, 256, 0, s>>>(acc, n_segments);
    int dev = 0, sms = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    k_noalloc_accumulate<<<2 * sms, 256, 0, s>>>((const uint4*)records, seg_offsets, n_segments, n_qubits, acc);
    k_noalloc_store<<<blocks_seg, 256, 0, s>>>(acc, n_segments, out);
    if (cudaGetLastError() != cudaSuccess) return QMC_ERR_CUDA;
    return QMC_OK;
}
