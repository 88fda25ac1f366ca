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

// records: 16-byte (uint64 key, int32 re, int32 im), keys (x << n) | y.
__global__ void k_noalloc_accumulate(const uint4* __restrict__ rec, const int64_t* __restrict__ off, int nseg, int n,
                                     ObsAcc* acc)
{
    const int64_t K = off[nseg];
    const uint32_t ymask = n == 32 ? 0xFFFFFFFFu : ((1u << n) - 1u);
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < K; i += (int64_t)gridDim.x * blockDim.x) {
        const uint4 r = rec[i];
        const uint64_t key = ((uint64_t)r.y << 32) | r.x;
        const int32_t re = (int32_t)r.z, im = (int32_t)r.w;
        const int s = seg_index(off, nseg, i);
        atomicAdd(&acc[s].count, 1ull);
        atomicAdd((unsigned long long*)&acc[s].ntot,
                  (unsigned long long)((re < 0 ? -(long long)re : re) + (im < 0 ? -(long long)im : im)));
        if ((uint32_t)(key >> n) == (uint32_t)(key & ymask)) {
            atomicAdd((unsigned long long*)&acc[s].dre, (unsigned long long)(long long)re);
            atomicAdd((unsigned long long*)&acc[s].dim, (unsigned long long)(long long)im);
        }
    }
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
    if (((uintptr_t)records & 15u) != 0) return QMC_ERR_INVALID_ARG;
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
