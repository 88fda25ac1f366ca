// Launch interface of the step for 33..60 qubits (library-internal).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "kernels.h"

namespace qmc {

// ---- the step for 33..60 qubits (128-bit keys, wide.cu) ----------------------
constexpr int kWMaxPasses = 20;      // 8-bit digits of (vector, key): up to 2 * 60 + 28 bits
constexpr int kWTile = 4096;         // records per tile of the radix sort's scatter
constexpr int kWChunk = 4096;        // extra draw calls (four walkers each) per heavy work item
constexpr int kWLight = 64;          // parents with more walkers take the heavy path
constexpr int kWScanTile = 2048;     // flags per tile of the new keys' prefix sums
constexpr int kWMTile = 4096;        // indices of N(t) per merge tile (index K: new keys after the last record)

// Run of equal (vector, key) in the sorted spawns, at its first record: the
// position of the key in N(t) (posA, a global index), whether N(t) holds it,
// and the sum of the spawns that survive the initiator rule (all of them
// when N(t) holds the key, the initiators' alone otherwise).
struct WRun {
    int64_t posA;
    int64_t re, im;
    int32_t matched, pad;
};


struct WideParams {
    WSpawn* spawn;          // unsorted spawns (sort ping-pong A)
    WSpawn* spawn_alt;      // sort ping-pong B
    WRun* run;              // [spawn_cap]
    int32_t* flag_u;        // [spawn_cap]: run head whose key is new to N(t + dt)
    int64_t* scan_u;        // [spawn_cap + 1]
    int2* delta;            // [pop_cap + 1]: per record of N(t) the spawn sum of the run on its key
                            //   (zero otherwise); zero between steps
    int32_t* newcnt;        // [pop_cap + 1]: new keys inserted just before record i; zero between steps
    int64_t* scan_a;        // [pop_cap + 2]: survivors of N(t) before record i, written where new keys
                            //   go just before i and at the first record of every vector
    unsigned long long* mtile;   // [mtiles_cap]: per merge tile, records the spawns zero | new keys << 32;
                                 //   zero between steps
    longlong2* mbase;       // [mtiles_cap]: per merge tile, survivors and new keys before it (last: totals)
    int64_t mtiles_cap;
    int64_t* abound;        // [2^kBucketBits + 1]: first record of N(t) in each bucket of the spawn sort
    uint32_t* win;          // [spawn_cap / 224 + 2]: start of each sort window of whole buckets
    uint32_t* big_list;     // [spawn_cap / 224 + 2]: windows too large for a warp
    uint32_t* nbig;         // how many of them (zeroed every step)
    int64_t* part;          // scan partials
    int64_t part_cap;
    uint32_t* hist;         // [kWMaxPasses][256] digit counts, then digit starts
    uint32_t* tile_hist;    // [tiles][256]
    int64_t tiles_cap;
    uint32_t* plan;         // [kWMaxPasses + 1]: per pass bit 0 skip, bit 1 source is spawn_alt; last: final buffer
    int passes;             // ceil((2n + vector bits) / 8)
};

void configure_wide_kernels();   // once per process, before the first capture of a wide step
// ev (optional): kNumWideGroups + 1 events; kernel group i runs between ev[i] and ev[i + 1].
constexpr int kNumWideGroups = 9;
extern const char* const kWideGroupNames[kNumWideGroups];
void launch_wide_step(const StepParams& P, const WideParams& W, cudaStream_t stream, cudaEvent_t* ev = nullptr);
int wide_step_launch_count(const StepParams& P, const WideParams& W);
void launch_wide_init(const StepParams& P, const uint64_t* xs, const uint64_t* ys, const double* re,
                      const double* im, int64_t nnz, int64_t* vals, cudaStream_t stream);
void launch_wide_obs(const StepParams& P, int which, SegStats* out, cudaStream_t stream);
void launch_wide_pack(const uint64_t* xs, const uint64_t* ys, const int32_t* re, const int32_t* im,
                      const int64_t* off, int nseg, const SegInfo* seginfo, uint8_t* dst, int64_t cap, int* bad,
                      cudaStream_t stream);
void launch_wide_lookup(const StepParams& P, int seg, const uint64_t* qx, const uint64_t* qy, int nq, int64_t* out,
                        cudaStream_t stream);
void launch_wide_export(const StepParams& P, int slot, int64_t first, int64_t count, uint64_t* x, uint64_t* y,
                        int32_t* re, int32_t* im, cudaStream_t stream);

} // namespace qmc
