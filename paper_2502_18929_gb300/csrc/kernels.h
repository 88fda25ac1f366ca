// Kernel launch interface (library-internal).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "qmc_types.h"

namespace qmc {

constexpr int kThreads = 256;
constexpr int kSortItems = 8;                        // records per thread per sort tile
constexpr int kSortTile = kThreads * kSortItems;     // 2048 records
constexpr int kMergeItems = 5;                       // 5 x 16 B stride: lanes spread over all bank groups
constexpr int kMergeTile = kThreads * kMergeItems;   // 1280 merged items
constexpr int kMergeThreads = kThreads + 64;         // merge CTA: 8 merging warps, a producer and a publisher
constexpr int kHeavyWalkers = 256;                   // default: parents above this take the heavy path
constexpr int64_t kHeavyChunk = 32768;               // walkers per heavy work item
constexpr int kMaxEntries = 1024;                    // destinations per column (heavy path)
constexpr int kMaxLearnedSlots = 256;                // destinations per column (learned proposal)
constexpr int kMaxHidden = 64;                       // hidden width of the learned proposal's network
constexpr int kMaxPasses = 12;
constexpr uint32_t kDefaultSpinLimit = 1u << 22;     // look-back polls before a wait gives up
constexpr int kBucketBits = 20;                    // largest bucket digit of the spawn sort
constexpr int kCtrMerge = kMaxPasses;                // tile counter index of the merge
constexpr int kCtrSpawn = kMaxPasses + 1;            // tile counter index of the light spawn
constexpr int kCtrBucket = kMaxPasses + 2;           // tile counter index of the bucket scan
constexpr uint32_t kTagStep = 0x53544550u;
constexpr uint32_t kTagInit = 0x494E4954u;
constexpr uint32_t kKindInit = 1u;
constexpr uint32_t kKindLearned = 2u;
constexpr uint32_t kKindGroup = 3u;     // spawn draws: first walkers of a rank group of four parents
constexpr uint32_t kKindExtra = 4u;     // spawn draws: further walkers of one parent, four per call
constexpr uint32_t kKindLow = 5u;       // spawn draws: the low 20 bits of one walker's T

struct HeavyItem {
    int64_t parent;  // index inside its population slot
    int32_t phase;   // 0: N(t), 1: N(t - dt)
    int32_t comp;    // 0: real walkers, 1: imaginary walkers
    int32_t chunk;   // walker chunk index
    int32_t seg;
};

// A walker whose 32-bit draw word W passes its program's prefilter (W <=
// P_bound >> 20): a spawn candidate, completed (T = W << 20 | L) and resolved
// against the exact column by k_spawn_choose.  16 bytes.
struct __align__(16) SpawnCand {
    uint32_t parent;  // index of the parent inside its population slot
    uint32_t seg;     // population vector
    uint32_t W;       // the walker's 32-bit draw word
    uint32_t meta;    // j (walker index in its component, 20 bits) | comp << 20 | phase << 21 |
                      // noninit << 22 | (parent component > 0) << 23
};

// One merge tile: its slices of the segment's N(t) records and sorted spawns,
// and the largest key before it (runs with that key belong to an earlier tile).
struct MTileG {
    int64_t a_glob;     // first N(t) record (index in the slot)
    int64_t b_glob;     // first spawn record (index in the sorted spawns)
    int64_t b_seg_end;  // end of the segment's spawns
    uint64_t prev_key;
    int32_t na, nb, seg, has_prev;
};

struct SegStats {
    unsigned long long count;
    long long ntot, dre, dim;
};

// Everything a step's kernels need.  Pointers are device pointers.
struct StepParams {
    DevState* st;
    const StepInfo* info;
    const uint8_t* progs;
    Rec* pop[3];
    int64_t* segoff[3];   // nseg + 1 offsets per slot
    int64_t* gofs[3];     // nseg + 1 rank-group offsets per slot (k_prologue, for N(t) and N(t - dt))
    int64_t pop_cap;
    SRec* spawn;          // spawn records (sort ping-pong A)
    SRec* spawn_alt;      // sort ping-pong B
    int64_t spawn_cap;
    SpawnCand* cand;      // spawn candidates of the step
    int64_t cand_cap;
    HeavyItem* heavy;
    int64_t heavy_cap;
    uint2* kd;            // per-segment Philox key of the current step
    unsigned int* sort_hist;   // [kMaxPasses][256]
    unsigned long long* sort_status; // [tiles][256] look-back words
    int64_t sort_tiles_cap;
    int64_t* bseg;        // nseg + 1: offsets of each segment in the sorted spawns
    int64_t* tile_start;  // nseg + 1: first merge tile of each segment
    MTileG* mtiles;       // per merge tile
    unsigned long long* merge_status; // per merge tile look-back word
    int64_t merge_tiles_cap;
    SegStats* segacc;     // per-segment accumulators of the merge
    SegStats* history;    // [steps of call][nseg]
    int64_t history_cap;  // steps
    long long* zacc;      // [nseg][32]: sum of Re N_xx over the diagonal records of N(t + dt) with bit q of x set
    long long* zhist;     // [steps of call][nseg][n]: sum over the diagonal of Re N_xx (-1)^(x_q)
    int n;                // largest qubit count of the instances (key width of the sorts)
    int nseg;
    int seg_bits;
    int key_passes;
    int seg_passes;
    int sort_mode;        // 0: LSD radix sort; 1: bucket pass + bucket sorts; 2: bucket pass alone
    int bucket_bits;      // bits of the bucket digit (<= kBucketBits)
    int bucket_kb;        // key bits in the bucket digit (below all segment bits)
    uint32_t spin_limit;  // polls of another CTA's look-back word before a wait gives up (0: none)
    uint32_t* bucket;     // 2^bucket_bits bucket counters / cursors
    unsigned long long* bscan_status; // look-back words of the bucket scan, 2^(kBucketBits - 10)
    uint32_t* big_list;   // buckets of the spawn sort too large for a lane
    const SegInfo* seginfo;   // per segment
    const InstInfo* inst;     // per instance
    int ninst;
    int proposal;         // 0: exact |L|-weighted destination choice; 1: static; 2: learned proposal
    const float* mlp;     // learned proposal: w1, b1, w2, b2, w3, b3 back to back
    int heavy_walkers;    // parents with more walkers take the heavy path
    const uint64_t* mlp_mask;   // output masks, sorted
    const int32_t* mlp_idx;     // output index of each sorted mask
    int mlp_in, mlp_hidden, mlp_out;
    float mlp_eps;
    const uint8_t* mlp_tc;   // the network for the tensor-core proposal (bf16 weights, padded; see TcLayout)
    int mlp_ip, mlp_gp;      // inputs padded to a multiple of 16, outputs to a multiple of 8
};

// The network in the tensor-core proposal's layout (bytes from the buffer's
// start): W1 [H][Ip + 8], W2 [H][H + 8], W3 [Gp][H + 8] in bf16 (row = output
// neuron, zero padding), then b1 [H], b2 [H], b3 [Gp] in fp32.  Rows are
// padded by 8 elements so that the eight rows a warp's B fragment reads fall
// in distinct shared-memory banks.
struct TcLayout {
    int I, H, G, Ip, Gp;
    int ld1, ld2, ld3;                 // row lengths (elements)
    int o_w1, o_w2, o_w3, o_b1, o_b2, o_b3, bytes;
};

__host__ __device__ inline TcLayout tc_layout(int I, int H, int G)
{
    TcLayout L;
    L.I = I;
    L.H = H;
    L.G = G;
    L.Ip = (I + 15) / 16 * 16;
    L.Gp = (G + 7) / 8 * 8;
    L.ld1 = L.Ip + 8;
    L.ld2 = H + 8;
    L.ld3 = H + 8;
    L.o_w1 = 0;
    L.o_w2 = L.o_w1 + 2 * H * L.ld1;
    L.o_w3 = L.o_w2 + 2 * H * L.ld2;
    L.o_b1 = (L.o_w3 + 2 * L.Gp * L.ld3 + 15) / 16 * 16;
    L.o_b2 = L.o_b1 + 4 * H;
    L.o_b3 = L.o_b2 + 4 * H;
    L.bytes = (L.o_b3 + 4 * L.Gp + 15) / 16 * 16;
    return L;
}

// Pack the fp32 parameters (w1, b1, w2, b2, w3, b3) into the tensor-core
// layout (bf16 weights rounded to nearest even).
void launch_mlp_tc_pack(const float* params, const TcLayout& L, uint8_t* out, cudaStream_t stream);

// Launchers (kernels.cu).  All take their sizes from DevState, so the same
// launch sequence can be captured once in a CUDA graph and replayed.
constexpr int kNumTimedKernels = 15;
void launch_learned_weights(const StepParams& P, bool tc, const uint8_t* prog, double t, const uint64_t* xs,
                            const uint64_t* ys, int count, int64_t* out, int cap, cudaStream_t stream);
void configure_kernels();  // once per process, before the first launch
extern const char* const kKernelNames[kNumTimedKernels];
void launch_step(const StepParams& P, int grid, cudaStream_t stream, cudaEvent_t* ev = nullptr);
int step_launch_count(const StepParams& P);   // kernels launch_step issues

// Training events of the learned proposal (learn.cu).  Device pointers.
struct LearnArgs {
    const DevState* st;
    Rec* pop[3];
    const uint8_t* prog;        // program of dt L(t) at the current time
    const uint64_t* masks;      // the network's output masks, sorted
    const int32_t* idx;         // output index of each sorted mask
    int n, G;
    double t;
    int64_t max_events, ld;
    float* feat;                // [2n + 1][ld]
    float* target;              // [G][ld]
    float* weight;              // [ld]
    int64_t* n_events;          // out: events written
};

// Loss and gradient of the learned proposal's network over events.
struct LearnGrad {
    const float* params;        // packed w1, b1, w2, b2, w3, b3
    const float* feat;
    const float* target;
    const float* weight;
    int64_t ld, E;
    int I, H, G;
    float *h1t, *h2t, *dzt, *d2t, *d1t, *lossv;   // scratch [rows][ld]
    double* wsum;
};

// Loss and gradient of the tensor-core proposal's network (bf16 operands,
// fp32 accumulation, GELU): one warp per 16 events for the forward pass, the
// masked softmax cross-entropy and the backpropagated signals (stored as bf16
// rows over events), then the weight gradients as bf16 matrix products over
// chunks of events, summed chunk by chunk in a fixed order.
struct LearnTc {
    const float* params;        // packed fp32 w1, b1, w2, b2, w3, b3 (master weights)
    const float* feat;
    const float* target;
    const float* weight;
    int64_t ld, E;              // the caller's event arrays: [rows][ld], E events
    int I, H, G;
    uint8_t* wts;               // training weights: TcLayout, then W2^T [H][H + 8], W3^T [H][Gp + 8] (bf16)
    int64_t ldp;                // scratch row length (E rounded up to 16)
    uint16_t *h1t, *h2t, *d1t, *d2t, *dzt;   // bf16 [rows][ldp]
    float* lossv;               // [ldp]
    float* partials;            // [chunks][params]
    double* wsum;
};
constexpr int64_t kLearnTcChunk = 4096;   // events per partial weight gradient
int64_t learn_tc_weights_bytes(int I, int H, int G);
int64_t learn_tc_scratch_bytes(int I, int H, int G, int64_t E);   // bf16 rows, losses and partials
void launch_learn_grad_tc(const LearnTc& A, float* grad, double* loss, cudaStream_t stream);

void launch_learn_events(const LearnArgs& A, cudaStream_t stream);
void launch_learn_grad(const LearnGrad& A, float* grad, double* loss, cudaStream_t stream);
int learn_grad_launch_count();
void launch_learn_adam(float* p, const float* g, float* m, float* v, int64_t n, int64_t t, float lr, float b1,
                       float b2, float eps, cudaStream_t stream);
void launch_pack(const uint64_t* keys, const int32_t* re, const int32_t* im, const int64_t* off, int nseg,
                 const SegInfo* seginfo, Rec* dst, int* bad, cudaStream_t stream);
void launch_obs(const StepParams& P, int which, SegStats* out, int grid, cudaStream_t stream);
void launch_lookup(const StepParams& P, int seg, const uint64_t* q, int nq, int64_t* out, cudaStream_t stream);
// Overlaps sum_ab conj(psi_a) N_ab psi_b of every vector of N(t) (out: nseg x (re, im)).
constexpr int kMaxOverlapLen = 64;
void launch_overlap_all(const StepParams& P, const uint64_t* idx, const double* psi, int len, double* out,
                        cudaStream_t stream);
// ||N - N^dagger||_F^2 of every vector of N(t), exactly (out: nseg x (low, high) 64-bit words, zeroed here).
void launch_antiherm(const StepParams& P, unsigned long long* out, int grid, cudaStream_t stream);
// ||S - S^dagger||_F^2 of the sum S of the listed vectors (device segs[count]); out: (low, high), zeroed here.
void launch_antiherm_sum(const StepParams& P, const int32_t* segs, int count, unsigned long long* out, int grid,
                         cudaStream_t stream);
void launch_init(const StepParams& P, const uint64_t* x, const uint64_t* y, const double* re, const double* im,
                 int64_t nnz, int64_t* tmp_vals, cudaStream_t stream);

} // namespace qmc
