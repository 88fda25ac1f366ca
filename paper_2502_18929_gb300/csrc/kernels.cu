// One step of real-time population-dynamics QMC on sm_103a (arXiv:2502.18929).
//
//   k_prologue      per-step Philox keys, counter resets
//   k_spawn_draw    walker draws [End Matter, spawn step] for parents with few
//                   walkers; draws below the bound on P become candidates
//   k_spawn_choose  exact spawn test and destination of every candidate
//   k_spawn_learned (learned proposal, in place of k_spawn_choose) the
//                   network's destination weights and the walker counts
//   k_spawn_heavy   the same for heavy parents, one CTA per walker chunk,
//                   aggregated per destination in shared memory
//                   (k_spawn_heavy_learned under the learned proposal)
//   k_sort_hist     digit histograms of all LSD radix passes
//   k_sort_scatter  one stable LSD pass, decoupled look-back, smem exchange
//   k_spawn_segoff  segment boundaries of the sorted spawns
//   k_merge_plan    merge tiles per segment
//   k_merge_part    merge-path partition of every tile
//   k_merge         annihilation [End Matter, annihilation step] + initiator
//                   rule + compaction + per-vector observables
//   k_finalize      segment offsets of N(t + dt), history, rotate the slots
//
// Integer-only: weights are exact 2^-52 fixed point, so spawning, annihilation
// and the observables are bit-identical to any other exact evaluation.  The
// learned proposal's network runs in single precision with each operation
// rounded explicitly, reproducible by a CPU that takes the same steps.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "column_eval.h"
#include "device_common.h"
#include "kernels.h"
#include "tc_ops.h"

namespace qmc {

namespace {

int g_grid_misc = 0;   // grid of the simple grid-stride kernels (set by configure_kernels)
constexpr uint32_t kFlagAgg = 1u, kFlagIncl = 2u;
// Polls of an mbarrier phase (a CTA's own bulk copies and its warps'
// hand-overs) before the wait gives up.  Waits on other CTAs' look-back words
// take the context's limit instead (StepParams::spin_limit).
constexpr uint32_t kMbarSpinLimit = 1u << 22;
constexpr int kStage = 64; // spawn records staged per warp

// A bounded wait that gave up: DERR_TIMEOUT, with the wait site and an index
// (tile or stage use) in error_aux for the host's message.
__device__ __forceinline__ void set_timeout(DevState* st, uint32_t site, int64_t idx)
{
    if (atomicCAS(&st->error, 0u, (uint32_t)DERR_TIMEOUT) == 0u)
        st->error_aux = (site << 24) | (uint32_t)(idx & 0xFFFFFF);
}

__device__ __forceinline__ unsigned long long ld_vol(const unsigned long long* p)
{
    return *(volatile const unsigned long long*)p;
}

__device__ __forceinline__ void st_vol(unsigned long long* p, unsigned long long v)
{
    *(volatile unsigned long long*)p = v;
}

// Look-back status word: epoch (26 bits) << 38 | flag (2 bits) << 36 | value
// (36 bits).  Epochs advance by 16 per step; the host clears the status
// arrays at least every 2^20 step launches, so a stale word never carries the
// current epoch.
constexpr unsigned long long kLbValMask = (1ull << 36) - 1ull;
constexpr uint32_t kLbEpochMask = (1u << 26) - 1u;

__device__ __forceinline__ unsigned long long lb_word(uint32_t epoch, uint32_t flag, unsigned long long v)
{
    return ((unsigned long long)(epoch & kLbEpochMask) << 38) | ((unsigned long long)flag << 36) | (v & kLbValMask);
}

__device__ __forceinline__ uint32_t lb_flag(unsigned long long v) { return (uint32_t)(v >> 36) & 3u; }

__device__ __forceinline__ bool lb_ready(unsigned long long v, uint32_t epoch)
{
    return (uint32_t)(v >> 38) == (epoch & kLbEpochMask) && lb_flag(v) != 0u;
}

// Wait (bounded) until *addr carries this epoch and a flag; returns false on
// timeout after raising DERR_TIMEOUT.
__device__ bool lb_wait(const unsigned long long* addr, uint32_t epoch, unsigned long long* out,
                        DevState* st, uint32_t site, int64_t idx, uint32_t limit)
{
    for (uint32_t it = 0; it < limit; ++it) {
        unsigned long long v = ld_vol(addr);
        if (lb_ready(v, epoch)) {
            *out = v;
            return true;
        }
        if (read_error(st) == DERR_TIMEOUT) break;
        if (it > 32) __nanosleep(64);
    }
    set_timeout(st, site, idx);
    return false;
}

// Warp-parallel decoupled look-back for tile t (all 32 lanes of one warp):
// lane i reads the status of tile t - 1 - i - 32 w in window w, the warp sums
// aggregates up to the nearest inclusive prefix.  Returns the exclusive
// prefix of tile t (to every lane).  Bounded waits; on timeout the error is
// raised and the partial sum returned.
__device__ unsigned long long warp_lookback(const unsigned long long* status, int64_t t, uint32_t epoch,
                                            DevState* st, int lane, uint32_t site, uint32_t limit)
{
    unsigned long long excl = 0;
    int64_t hi = t - 1; // nearest unread predecessor
    while (hi >= 0) {
        const int64_t j = hi - lane;
        unsigned long long v = 0;
        bool ready = j < 0;
        for (uint32_t it = 0; it < limit; ++it) {
            if (!ready) {
                v = ld_vol(status + j);
                ready = lb_ready(v, epoch);
            }
            if (__all_sync(kFull, ready)) break;
            if (read_error(st) == DERR_TIMEOUT) break;
            if (it > 32) __nanosleep(64);
        }
        if (!__all_sync(kFull, ready)) {
            if (lane == 0) set_timeout(st, site, t);
            break;
        }
        const bool incl = j >= 0 && lb_flag(v) == kFlagIncl;
        const uint32_t bal = __ballot_sync(kFull, incl);
        const int stop = bal ? __ffs(bal) - 1 : 31;          // lanes 0..stop contribute
        unsigned long long c = (j >= 0 && lane <= stop) ? (v & kLbValMask) : 0ull;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(kFull, c, o);
        excl += c;
        if (bal) break;
        hi -= 32;
    }
    return excl;
}

// The record of one spawned walker.  sign rule [End Matter, spawn step]:
// Re channel s sgn(Re L), Im channel i s sgn(Im L); s = sgn(re) for a real
// walker, i sgn(im) for an imaginary one; sigma = -1 for the N(t - dt) pass.
__device__ __forceinline__ SRec make_spawn(uint64_t dest, int seg, int comp, int chan, int64_t v,
                                           int sg, int sigma, int noninit, int32_t count)
{
    const int s = sigma * sg * (v > 0 ? 1 : -1);
    int target, val;
    if (chan == 0) { target = comp; val = s; }
    else if (comp == 0) { target = 1; val = s; }
    else { target = 0; val = -s; }
    SRec r;
    r.key = dest;
    r.meta = ((uint32_t)seg << 2) | ((uint32_t)target << 1) | (uint32_t)noninit;
    r.val = val * count;
    return r;
}

// ---------------------------------------------------------------------------
// Prologue: keys of this step, counter resets.
// ---------------------------------------------------------------------------
__global__ void k_prologue(StepParams P)
{
    DevState* st = P.st;
    if (read_error(st)) return;
    const uint64_t step = st->step;
    for (int s = threadIdx.x; s < P.nseg; s += blockDim.x) {
        const SegInfo si = P.seginfo[s];
        const uint64_t seed = P.inst[si.inst].seed;
        uint4 o = philox10(make_uint4((uint32_t)step, (uint32_t)(step >> 32), (uint32_t)si.vec, kTagStep),
                           make_uint2((uint32_t)seed, (uint32_t)(seed >> 32)));
        P.kd[s] = make_uint2(o.x, o.y);
        P.segacc[s] = SegStats{0ull, 0ll, 0ll, 0ll};
    }
    for (int64_t i = threadIdx.x; i < 32 * (int64_t)P.nseg; i += blockDim.x) P.zacc[i] = 0ll;
    for (int i = threadIdx.x; i < kMaxPasses * 256; i += blockDim.x) P.sort_hist[i] = 0u;
    for (int i = threadIdx.x; i < kMaxTileCounters; i += blockDim.x) st->tile_ctr[i] = 0u;
    // rank-group offsets of N(t) and N(t - dt) (the draw kernel's work units):
    // gof[s] = sum over the vectors before s of ceil(K / 4)
    __shared__ long long wsum[kThreads / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int w = 0; w < 2; ++w) {
        const int slot = w ? (st->cur + 2) % 3 : st->cur;
        const int64_t* off = P.segoff[slot];
        int64_t* gof = P.gofs[slot];
        long long carry = 0;
        for (int base = 0; base < P.nseg; base += kThreads) {
            const int s = base + threadIdx.x;
            const long long c = s < P.nseg ? (long long)((off[s + 1] - off[s] + 3) / 4) : 0ll;
            long long incl = c;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const long long v = __shfl_up_sync(kFull, incl, o);
                if (lane >= o) incl += v;
            }
            if (lane == 31) wsum[warp] = incl;
            __syncthreads();
            long long wo = 0, blk = 0;
            for (int q = 0; q < kThreads / 32; ++q) {
                if (q < warp) wo += wsum[q];
                blk += wsum[q];
            }
            if (s < P.nseg) gof[s] = carry + wo + incl - c;
            carry += blk;
            __syncthreads();
        }
        if (threadIdx.x == 0) gof[P.nseg] = carry;
    }
    if (threadIdx.x == 0) {
        st->spawn_total = 0;
        st->cand_total = 0;
        // LSD radix sort when the bucket sort does not apply (it may still fall back to it)
        st->sort_fallback = P.sort_mode == 0 ? 1u : 0u;
        st->big_windows = 0u;
        st->sort_final = P.sort_mode == 0 ? (uint32_t)((P.key_passes + P.seg_passes) & 1) : 1u;
        st->heavy_total = 0;
        st->next_total = 0;
        st->merge_tiles = 0;
        st->seq += 16u;
    }
}

// ---------------------------------------------------------------------------
// Spawning, light parents [End Matter, spawn step], in two kernels.
//   k_spawn_draw: a warp takes rank groups of four consecutive parents, one
//     group per lane: one Philox call gives the 32-bit draw words W of the
//     four parents' first walkers, further walkers take four words per call
//     of their parent; a walker whose W passes the program's prefilter
//     (W <= P_bound >> 20) becomes a candidate.  Parents with many walkers
//     become heavy work items.
//   k_spawn_choose: one thread per candidate completes the walker's draw
//     T = W << 20 | L (52 bits), evaluates the exact weight P of the
//     parent's column; the walker spawns iff T < P, onto the destination
//     whose cumulative-weight interval holds T (canonical order).
// ---------------------------------------------------------------------------
constexpr int kProgSmem = 8192;

__device__ __forceinline__ void warp_flush(SRec* stage, int n, const StepParams& P, int lane)
{
    unsigned long long base = 0;
    if (lane == 0) base = atomicAdd((unsigned long long*)&P.st->spawn_total, (unsigned long long)n);
    base = __shfl_sync(kFull, base, 0);
    if ((int64_t)base + n > P.spawn_cap) {
        if (lane == 0) set_error(P.st, DERR_SPAWN_CAPACITY);
    }
    for (int j = lane; j < n; j += 32) {
        const int64_t pos = (int64_t)base + j;
        if (pos < P.spawn_cap) P.spawn[pos] = stage[j];
    }
    __syncwarp();
}

// Copy a program into shared memory if it fits; returns the copy to use once
// the block has synchronised (the caller must __syncthreads() before reading).
__device__ __forceinline__ const uint8_t* stage_prog(const uint8_t* g, uint8_t* s)
{
    const int bytes = ((const ProgHeader*)g)->bytes;
    if (bytes > kProgSmem) return g;
    for (int i = threadIdx.x; i < bytes / 8; i += blockDim.x)
        ((uint64_t*)s)[i] = ((const uint64_t*)g)[i];
    return s;
}

// ---------------------------------------------------------------------------
// Bulk (TMA) copies into shared memory, completed on an mbarrier.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_addr(const void* p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_fence_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void fence_proxy_async()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect(uint64_t* bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}

// 1-D bulk copy global -> shared; both addresses 16-byte aligned, bytes a
// multiple of 16.
__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_addr(dst)),
                 "l"(src), "r"(bytes), "r"(smem_addr(bar))
                 : "memory");
}

__device__ __forceinline__ bool mbar_try(uint64_t* bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
                 : "=r"(ok)
                 : "r"(smem_addr(bar)), "r"(parity)
                 : "memory");
    return ok != 0;
}

// Bounded wait for a phase of an mbarrier.
__device__ bool mbar_wait(uint64_t* bar, uint32_t parity, DevState* st, uint32_t site, int64_t idx)
{
    for (uint32_t it = 0; it < kMbarSpinLimit; ++it) {
        if (mbar_try(bar, parity)) return true;
        if (it > 16) __nanosleep(32);
    }
    set_timeout(st, site, idx);
    return false;
}

constexpr int kCandStage = 256;   // candidates staged per warp
constexpr int kCandFlush = 128;   // a warp flushes once more than this are staged
constexpr uint32_t kJ20 = (1u << 20) - 1u;

// Append a warp's staged candidates to the candidate list of the step.
__device__ __forceinline__ void cand_flush(const SpawnCand* stage, int n, const StepParams& P, int lane)
{
    unsigned long long base = 0;
    if (lane == 0) base = atomicAdd((unsigned long long*)&P.st->cand_total, (unsigned long long)n);
    base = __shfl_sync(kFull, base, 0);
    if ((int64_t)base + n > P.cand_cap && lane == 0) set_error(P.st, DERR_CAND_CAPACITY);
    const uint4* s4 = (const uint4*)stage;
    uint4* d4 = (uint4*)P.cand;
    for (int j = lane; j < n; j += 32) {
        const int64_t pos = (int64_t)base + j;
        if (pos < P.cand_cap) d4[pos] = s4[j];
    }
    __syncwarp();
}

// Candidate word w: the walker's index j in its component (20 bits), the
// component, the pass, the initiator flag and the sign of the parent's
// component (SpawnCand).
__device__ __forceinline__ uint32_t cand_meta(uint32_t j, int comp, int phase, int noninit, int32_t val)
{
    return j | ((uint32_t)comp << 20) | ((uint32_t)phase << 21) | ((uint32_t)noninit << 22) |
           ((uint32_t)(val > 0 ? 1 : 0) << 23);
}

// Emit the heavy work items of one parent (one per kHeavyChunk walkers of
// each component).
__device__ void emit_heavy(const StepParams& P, int64_t parent, int phase, int seg, uint32_t are, uint32_t aim)
{
    for (int comp = 0; comp < 2; ++comp) {
        const int64_t m = comp ? aim : are;
        const int64_t chunks = (m + kHeavyChunk - 1) / kHeavyChunk;
        if (chunks == 0) continue;
        const unsigned long long hb = atomicAdd((unsigned long long*)&P.st->heavy_total, (unsigned long long)chunks);
        for (int64_t c = 0; c < chunks; ++c) {
            const int64_t pos = (int64_t)hb + c;
            if (pos < P.heavy_cap) {
                HeavyItem h;
                h.parent = parent;
                h.phase = phase;
                h.comp = comp;
                h.chunk = (int32_t)c;
                h.seg = seg;
                P.heavy[pos] = h;
            } else {
                set_error(P.st, DERR_HEAVY_CAPACITY);
            }
        }
    }
}

// Column program of one instance for one pass of the current step.
__device__ __forceinline__ const uint8_t* prog_ptr(const StepParams& P, const StepInfo& inf, int inst, int phase)
{
    const int64_t* tab = (const int64_t*)(P.progs + inf.tab_off);
    return P.progs + tab[2 * inst + phase];
}

// Draw parameters of one vector in one pass of the current step: its Philox
// key, the prefilter bound on a walker's 32-bit word W (T = W << 20 | L < P
// needs W <= P >> 20; all: every walker is a candidate, the bound having
// reached 2^52), and its instance's initiator threshold.
struct SegDraw {
    uint32_t pre;        // W <= pre: candidate (2^32 - 1 once the bound reaches 2^52: every walker)
    uint32_t init_thr;   // parents with fewer walkers are non-initiators (0: none)
    uint2 kd;
};

__device__ __forceinline__ SegDraw seg_draw(const StepParams& P, const StepInfo& inf, int seg, int phase)
{
    const SegInfo si = P.seginfo[seg];
    const ProgHeader* h = (const ProgHeader*)prog_ptr(P, inf, si.inst, phase);
    const int64_t pb = P.proposal ? h->p_att : h->p_bound;   // attempt bound of the choice rule
    const int64_t im = P.inst[si.inst].init_min;
    SegDraw d;
    d.pre = pb >= (1ll << 52) ? 0xFFFFFFFFu : (uint32_t)(pb >> 20);
    d.init_thr = im <= 0 ? 0u : (im >= 0xFFFFFFFFll ? 0xFFFFFFFFu : (uint32_t)im);
    d.kd = P.kd[seg];
    return d;
}

__device__ __forceinline__ bool passes(const SegDraw& d, uint32_t W) { return W <= d.pre; }

// Vector holding group G of a slot: the largest s with gof[s] <= G (s = nseg
// for G = the slot's group count).
__device__ __forceinline__ int group_seg(const int64_t* gof, int nseg, int64_t G)
{
    int lo = 0, hi = nseg;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (__ldg(&gof[mid]) <= G) lo = mid; else hi = mid - 1;
    }
    return lo;
}

constexpr int kDrawGroups = 32;                 // rank groups per warp iteration, one per lane
constexpr int kDrawRecs = 4 * kDrawGroups;      // records staged per iteration (2 KB)
constexpr int kDrawStages = 3;                  // staged iterations per warp
constexpr int kDrawWarps = kThreads / 32;
constexpr int kXRing = 256;                     // queued single-call parents per warp (a power of two)
constexpr int kDrawSmem = kDrawWarps * (kDrawStages * kDrawRecs * 16 + kCandStage * 16 + kXRing * 16);

__device__ __forceinline__ uint32_t uabs32(int32_t v) { return v < 0 ? 0u - (uint32_t)v : (uint32_t)v; }

// Warp-wide placement of up to four items per lane (bit i of `bits`): one
// ballot per slot i; slot i's items follow slot i - 1's, lanes in order.
// Returns the total; off[i] is the lane's position for its slot-i item.
__device__ __forceinline__ int warp_place4(uint32_t bits, int (&off)[4], int lane)
{
    const uint32_t lt = (1u << lane) - 1u;
    int base = 0;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const uint32_t b = __ballot_sync(kFull, (bits >> i) & 1u);
        off[i] = base + __popc(b & lt);
        base += __popc(b);
    }
    return base;
}

// Make room for `tot` more candidates in the warp's stage (flushing it first
// if needed); returns the stage position where they start.
__device__ __forceinline__ int cand_reserve(SpawnCand* stage, int* staged, int tot, const StepParams& P, int lane)
{
    if (*staged + tot > kCandStage) {
        cand_flush(stage, *staged, P, lane);
        *staged = 0;
    }
    const int at = *staged;
    *staged += tot;
    return at;
}

__device__ __forceinline__ void cand_done(SpawnCand* stage, int* staged, const StepParams& P, int lane)
{
    __syncwarp();
    if (*staged > kCandFlush) {
        cand_flush(stage, *staged, P, lane);
        *staged = 0;
    }
}

// Candidates among the walkers 2 + 4b .. 5 + 4b of one parent (its call b):
// staged for the lanes that are active.  Whole warp.
__device__ __forceinline__ void extra_draw(SpawnCand* stage, int* staged, const StepParams& P, const SegDraw& d,
                                           uint32_t parent, uint32_t seg, uint32_t rank, uint32_t b, int32_t re,
                                           int32_t im, int phase, bool act, int lane)
{
    const uint32_t are = uabs32(re), m = are + uabs32(im);
    const uint4 xw = extra_words(rank, b, phase, d.kd);
    uint32_t bits = 0u;
#pragma unroll
    for (int q = 0; q < 4; ++q)
        if (act && 2u + 4u * b + (uint32_t)q < m && passes(d, word_of(xw, q))) bits |= 1u << q;
    int off[4];
    const int tot = warp_place4(bits, off, lane);
    if (tot == 0) return;
    const int at = cand_reserve(stage, staged, tot, P, lane);
    if (bits) {
        const uint32_t noninit = m < d.init_thr ? 1u : 0u;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            if (!((bits >> q) & 1u)) continue;
            const uint32_t w = 2u + 4u * b + (uint32_t)q;
            const int comp = w < are ? 0 : 1;
            ((uint4*)stage)[at + off[q]] =
                make_uint4(parent, seg, word_of(xw, q),
                           cand_meta(comp ? w - are : w, comp, phase, (int)noninit, comp ? im : re));
        }
    }
    cand_done(stage, staged, P, lane);
}

// Walker draws of one population slot (phase 0: N(t), phase 1: N(t - dt)).
// The slot's records form rank groups of four consecutive records of one
// vector (the last group of a vector may be shorter); the warp owns groups
// [gb, ge) and takes them 32 at a time, lane l group G0 + l, their records
// staged by one bulk copy per iteration (kDrawStages - 1 iterations ahead).
// A lane draws its group call (one Philox call: the first walkers of its four
// parents) and compares each word with the vector's prefilter bound; the
// group's level-1 call gives the second walkers.  Parents with 3 to 6
// walkers (one further call) are queued per warp and their calls drawn 32 at
// a time; parents with 7 to heavy_walkers walkers take their calls at once,
// spread evenly over the lanes; heavier parents become heavy work items (all
// their walkers).  Record indices and walker
// counts fit 32 bits (at most 2^31 - 1 records per slot, |re|, |im| < 2^31).
__device__ __forceinline__ void draw_slot(const StepParams& P, SpawnCand* stage, int* staged, uint4* xring,
                                          int* xhead, int* xcnt, Rec* buf, uint64_t* bar, uint32_t* use_no,
                                          const Rec* src, const int64_t* off, const int64_t* gof, int64_t gb,
                                          int64_t ge, int phase, const StepInfo& inf, int lane)
{
    const int nseg = P.nseg;
    const int64_t Gt = gof[nseg];
    const int64_t nit = (ge - gb + kDrawGroups - 1) / kDrawGroups;
    const uint32_t u0 = *use_no;
    const uint32_t heavy_w = (uint32_t)P.heavy_walkers;
    bool gave_up = false;
    // lane 0: a cursor over the slot's vectors for the copies issued ahead
    // (the iterations' record ranges follow one another)
    int cs = 0;
    int64_t c_gof = 0, c_gend = 0, c_off = 0, next_r = 0;
    if (lane == 0 && nit > 0) {
        cs = group_seg(gof, nseg, gb);
        c_gof = __ldg(&gof[cs]);
        c_gend = __ldg(&gof[cs + 1]);
        c_off = __ldg(&off[cs]);
        next_r = c_off + 4 * (gb - c_gof);
    }
    auto rec_at = [&](int64_t B) -> int64_t {   // first record of group B (B > the last one asked)
        if (B >= Gt) return __ldg(&off[nseg]);
        while (B >= c_gend) {
            ++cs;
            c_gof = c_gend;
            c_gend = __ldg(&gof[cs + 1]);
            c_off = __ldg(&off[cs]);
        }
        return c_off + 4 * (B - c_gof);
    };
    // lane 0: bulk copy of iteration k's records into stage (u0 + k) % kDrawStages
    auto issue = [&](int64_t k) {
        const uint32_t u = u0 + (uint32_t)k;
        const int64_t B = min(ge, gb + (k + 1) * kDrawGroups);
        const int64_t r0 = next_r, r1 = rec_at(B);
        next_r = r1;
        const uint32_t bytes = (uint32_t)(r1 - r0) * 16u;
        uint64_t* b = bar + u % kDrawStages;
        fence_proxy_async();
        mbar_arrive_expect(b, bytes);
        bulk_load(buf + (u % kDrawStages) * kDrawRecs, src + r0, bytes, b);
    };
    // the queued parents' calls, 32 at a time (n <= 32 entries from the head)
    auto drain = [&](int n) {
        const bool act = lane < n;
        const uint4 e = act ? xring[(*xhead + lane) & (kXRing - 1)] : make_uint4(0u, 0u, 0u, 0u);
        SegDraw d;
        d.pre = 0u;
        d.init_thr = 0u;
        d.kd = make_uint2(0u, 0u);
        uint32_t rank = 0u;
        if (act) {
            d = seg_draw(P, inf, (int)e.y, phase);
            rank = e.x - (uint32_t)__ldg(&off[e.y]);
        }
        extra_draw(stage, staged, P, d, e.x, e.y, rank, 0u, (int32_t)e.z, (int32_t)e.w, phase, act, lane);
        *xhead = (*xhead + n) & (kXRing - 1);
        *xcnt -= n;
    };
    if (lane == 0)
        for (int64_t k = 0; k < kDrawStages - 1 && k < nit; ++k) issue(k);
    // the lane's vector (cached while its groups stay inside it)
    int seg = 0;
    int64_t seg_gend = -1;
    uint32_t seg_off = 0u, seg_gof = 0u, seg_K = 0u;
    SegDraw sd;
    sd.pre = 0u;
    sd.init_thr = 0u;
    sd.kd = make_uint2(0u, 0u);
    for (int64_t k = 0; k < nit; ++k) {
        const uint32_t u = u0 + (uint32_t)k;
        const int64_t G0 = gb + k * kDrawGroups;
        const int64_t Gend = min(ge, G0 + kDrawGroups);
        if (lane == 0 && k + kDrawStages - 1 < nit) issue(k + kDrawStages - 1);
        const Rec* tb = buf + (u % kDrawStages) * kDrawRecs;
        const bool ok = mbar_wait(bar + u % kDrawStages, (u / kDrawStages) & 1u, P.st, 7u, k);
        if (!ok) gave_up = true;
        const int64_t G = G0 + lane;
        const bool valid = ok && G < Gend;
        if (valid && G >= seg_gend) {
            seg = group_seg(gof, nseg, G);
            seg_gend = __ldg(&gof[seg + 1]);
            seg_off = (uint32_t)__ldg(&off[seg]);
            seg_gof = (uint32_t)__ldg(&gof[seg]);
            seg_K = (uint32_t)__ldg(&off[seg + 1]) - seg_off;
            sd = seg_draw(P, inf, seg, phase);
        }
        const uint32_t g = (uint32_t)G - seg_gof;
        const uint32_t first = seg_off + 4u * g;
        const uint32_t rem = seg_K - 4u * g;
        const int cnt = valid ? (rem < 4u ? (int)rem : 4) : 0;
        // the stage starts at the first record of group G0, lane 0's
        const uint32_t r0 = __shfl_sync(kFull, first, 0);
        const int pos = (int)(first - r0);
        const uint4 gw = group_words(g, 0u, phase, sd.kd);
        int32_t re[4], im[4];
        uint32_t pass = 0u, two = 0u, queue = 0u, multi = 0u, heavy = 0u;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            re[i] = 0;
            im[i] = 0;
            if (i < cnt) {
                const uint4 w = ((const uint4*)tb)[pos + i];
                re[i] = (int32_t)w.z;
                im[i] = (int32_t)w.w;
            }
            const uint32_t m = uabs32(re[i]) + uabs32(im[i]);
            if (i < cnt) {
                if (m > heavy_w) heavy |= 1u << i;
                else {
                    if (passes(sd, word_of(gw, i))) pass |= 1u << i;
                    if (m >= 2u) two |= 1u << i;
                    if (m >= 3u) {
                        if (m <= 6u) queue |= 1u << i;
                        else multi |= 1u << i;
                    }
                }
            }
        }
        if (__any_sync(kFull, heavy != 0u)) {
#pragma unroll
            for (int i = 0; i < 4; ++i)
                if ((heavy >> i) & 1u) emit_heavy(P, first + i, phase, seg, uabs32(re[i]), uabs32(im[i]));
        }
        // the first walkers that pass: staged
        {
            int offs[4];
            const int tot = warp_place4(pass, offs, lane);
            if (tot) {
                const int at = cand_reserve(stage, staged, tot, P, lane);
                if (pass) {
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        if (!((pass >> i) & 1u)) continue;
                        const uint32_t m = uabs32(re[i]) + uabs32(im[i]);
                        const int comp = re[i] ? 0 : 1;
                        ((uint4*)stage)[at + offs[i]] =
                            make_uint4(first + i, (uint32_t)seg, word_of(gw, i),
                                       cand_meta(0u, comp, phase, m < sd.init_thr ? 1 : 0, comp ? im[i] : re[i]));
                    }
                }
                cand_done(stage, staged, P, lane);
            }
        }
        // the second walkers: the rank group's level-1 call
        if (__any_sync(kFull, two != 0u)) {
            const uint4 gw1 = group_words(g, 1u, phase, sd.kd);
            uint32_t pass1 = 0u;
#pragma unroll
            for (int i = 0; i < 4; ++i)
                if (((two >> i) & 1u) && passes(sd, word_of(gw1, i))) pass1 |= 1u << i;
            int offs[4];
            const int tot = warp_place4(pass1, offs, lane);
            if (tot) {
                const int at = cand_reserve(stage, staged, tot, P, lane);
                if (pass1) {
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        if (!((pass1 >> i) & 1u)) continue;
                        const uint32_t are = uabs32(re[i]), m = are + uabs32(im[i]);
                        const int comp = 1u < are ? 0 : 1;
                        ((uint4*)stage)[at + offs[i]] =
                            make_uint4(first + i, (uint32_t)seg, word_of(gw1, i),
                                       cand_meta(comp ? 1u - are : 1u, comp, phase, m < sd.init_thr ? 1 : 0,
                                                 comp ? im[i] : re[i]));
                    }
                }
                cand_done(stage, staged, P, lane);
            }
        }
        // queue the parents with 3 to 6 walkers: walkers 2 .. 5 in one call (drawn 32 calls at a time)
        {
            int offs[4];
            const int tot = warp_place4(queue, offs, lane);
            if (tot) {
                const int tail = *xhead + *xcnt;
#pragma unroll
                for (int i = 0; i < 4; ++i)
                    if ((queue >> i) & 1u)
                        xring[(tail + offs[i]) & (kXRing - 1)] =
                            make_uint4(first + i, (uint32_t)seg, (uint32_t)re[i], (uint32_t)im[i]);
                *xcnt += tot;
                __syncwarp();
                while (*xcnt >= 32) {
                    drain(32);
                    __syncwarp();
                }
            }
        }
        // parents with 7 .. heavy_walkers walkers: their calls at once, spread evenly over the lanes
        if (__any_sync(kFull, multi != 0u)) {
            int ne[4];
            int total_ne = 0;
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                ne[i] = ((multi >> i) & 1u) ? (int)((uabs32(re[i]) + uabs32(im[i]) + 1u) / 4u) : 0;
                total_ne += ne[i];
            }
            int incl = total_ne;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int t = __shfl_up_sync(kFull, incl, o);
                if (lane >= o) incl += t;
            }
            const int tot = __shfl_sync(kFull, incl, 31);
            for (int rr = 0; rr < tot; rr += 32) {
                const int gi = rr + lane;
                int lo = 0, hi = 31;   // owner: the first lane whose inclusive count exceeds gi
                while (lo < hi) {
                    const int mid = (lo + hi) >> 1;
                    if (__shfl_sync(kFull, incl, mid) > gi) hi = mid; else lo = mid + 1;
                }
                const int owner = lo;
                const bool act = gi < tot;
                int local = gi - (__shfl_sync(kFull, incl, owner) - __shfl_sync(kFull, total_ne, owner));
                int o_ne[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) o_ne[q] = __shfl_sync(kFull, ne[q], owner);
                const int o_pos = __shfl_sync(kFull, pos, owner);
                const uint32_t o_first = __shfl_sync(kFull, first, owner);
                const int o_seg = __shfl_sync(kFull, seg, owner);
                const uint32_t o_g = __shfl_sync(kFull, g, owner);
                SegDraw od;
                od.kd = make_uint2(__shfl_sync(kFull, sd.kd.x, owner), __shfl_sync(kFull, sd.kd.y, owner));
                od.pre = __shfl_sync(kFull, sd.pre, owner);
                od.init_thr = __shfl_sync(kFull, sd.init_thr, owner);
                int i = 0;   // the owner's parent holding call `local`, then the call's index in it
#pragma unroll
                for (int q = 0; q < 3; ++q) {
                    if (i == q && local >= o_ne[q]) {
                        local -= o_ne[q];
                        ++i;
                    }
                }
                int32_t pre_ = 0, pim = 0;
                if (act) {
                    const uint4 w = ((const uint4*)tb)[o_pos + i];
                    pre_ = (int32_t)w.z;
                    pim = (int32_t)w.w;
                }
                extra_draw(stage, staged, P, od, o_first + (uint32_t)i, (uint32_t)o_seg, 4u * o_g + (uint32_t)i,
                           (uint32_t)local, pre_, pim, phase, act, lane);
            }
        }
        __syncwarp();   // every read of the stage done before it is refilled
    }
    if (*xcnt > 0) {
        drain(*xcnt);
        __syncwarp();
    }
    if (gave_up) {
        // a copy may still be landing in the last stages: wait for them once more (bounded)
        for (int64_t k = nit > kDrawStages ? nit - kDrawStages : 0; k < nit; ++k) {
            const uint32_t u = u0 + (uint32_t)k;
            mbar_wait(bar + u % kDrawStages, (u / kDrawStages) & 1u, P.st, 7u, k);
        }
    }
    *use_no = u0 + (uint32_t)nit;
}

__global__ void __launch_bounds__(kThreads, 2) k_spawn_draw(StepParams P)
{
    extern __shared__ __align__(128) uint4 dsm[];
    __shared__ __align__(8) uint64_t sbar[kDrawWarps][kDrawStages];
    DevState* st = P.st;
    if (cta_error(st)) return;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    Rec* buf = (Rec*)(dsm + warp * (kDrawStages * kDrawRecs));
    SpawnCand* stage = (SpawnCand*)(dsm + kDrawWarps * kDrawStages * kDrawRecs + warp * kCandStage);
    uint4* xring = dsm + kDrawWarps * (kDrawStages * kDrawRecs + kCandStage) + warp * kXRing;
    int xhead = 0, xcnt = 0;
    if (P.sort_mode)   // bucket counters of this step's spawn sort
        for (int b = blockIdx.x * kThreads + threadIdx.x; b < (1 << P.bucket_bits); b += gridDim.x * kThreads)
            P.bucket[b] = 0u;
    if (lane == 0) {
        for (int q = 0; q < kDrawStages; ++q) mbar_init(&sbar[warp][q], 1);
        mbar_fence_init();
    }
    __syncwarp();
    uint32_t use_no = 0;
    const StepInfo inf = P.info[st->call_index];
    const int cur = st->cur, prv = (cur + 2) % 3;
    const int64_t nwarps = (int64_t)gridDim.x * kDrawWarps;
    const int64_t gw = (int64_t)blockIdx.x * kDrawWarps + warp;
    int staged = 0;
    for (int phase = 0; phase < (inf.ab2 ? 2 : 1); ++phase) {
        const int slot = phase ? prv : cur;
        const int64_t* gof = P.gofs[slot];
        const int64_t Gt = gof[P.nseg];
        // each warp owns one contiguous range of the slot's rank groups, a multiple of 32
        const int64_t chunk = ((Gt + nwarps - 1) / nwarps + kDrawGroups - 1) / kDrawGroups * kDrawGroups;
        const int64_t gb = min(Gt, gw * chunk), ge = min(Gt, gb + chunk);
        draw_slot(P, stage, &staged, xring, &xhead, &xcnt, buf, sbar[warp], &use_no, P.pop[slot], P.segoff[slot], gof,
                  gb, ge, phase, inf, lane);
    }
    if (staged) cand_flush(stage, staged, P, lane);
}

// One thread per candidate: exact weight P of the parent's column, the spawn
// test T < P, and the destination.  Programs are staged in shared memory.
__global__ void __launch_bounds__(kThreads, 3) k_spawn_choose(StepParams P)
{
    __shared__ __align__(16) uint8_t sprog[2][kProgSmem];
    __shared__ __align__(16) SRec sstage[kThreads / 32][kStage];
    DevState* st = P.st;
    if (cta_error(st)) return;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const StepInfo inf = P.info[st->call_index];
    const int cur = st->cur, prv = (cur + 2) % 3;
    const Rec* src0 = P.pop[cur];
    const Rec* src1 = P.pop[prv];
    // one instance: its two programs staged in shared memory; several: each
    // candidate reads its instance's program from global memory (L2-resident)
    const bool single = P.ninst == 1;
    const uint8_t* pb0 = single ? stage_prog(prog_ptr(P, inf, 0, 0), sprog[0]) : nullptr;
    const uint8_t* pb1 = single ? stage_prog(prog_ptr(P, inf, 0, inf.ab2 ? 1 : 0), sprog[1]) : nullptr;
    __syncthreads();   // programs staged
    const int64_t total = min(st->cand_total, P.cand_cap);
    SRec* stage = sstage[warp];
    int staged = 0;
    const int64_t stride = (int64_t)gridDim.x * kThreads;
    for (int64_t base = (int64_t)blockIdx.x * kThreads + warp * 32; base < total; base += stride) {
        const int64_t i = base + lane;
        SRec rec;
        bool ok = false;
        if (i < total) {
            const uint4 cv = __ldcs((const uint4*)P.cand + i);
            const int comp = (int)((cv.w >> 20) & 1u), phase = (int)((cv.w >> 21) & 1u);
            const int non = (int)((cv.w >> 22) & 1u), sg = ((cv.w >> 23) & 1u) ? 1 : -1;
            // the walker's full draw from its rank in the vector
            const uint32_t rank = cv.x - (uint32_t)__ldg(&P.segoff[phase ? prv : cur][cv.y]);
            const int64_t T = walker_T(cv.z, rank, cv.w & kJ20, comp, phase, P.kd[cv.y]);
            const uint64_t key = __ldg(&(phase ? src1 : src0)[cv.x].key);
            const SegInfo si = P.seginfo[cv.y];
            const int n = si.n;
            const uint32_t x = (uint32_t)(key >> n), y = (uint32_t)(key & (n == 32 ? 0xFFFFFFFFu : ((1u << n) - 1u)));
            const Prog prog = prog_at(single ? (phase ? pb1 : pb0) : prog_ptr(P, inf, si.inst, phase));
            if (P.proposal) {
                // static-weight proposal: every candidate is an attempt (T < p_att)
                uint64_t mk;
                int chan;
                int64_t v;
                if (prog.h->p_att >= (1ll << 52)) set_error(st, DERR_DT_TOO_LARGE);
                else if (T < prog.h->p_att && proposal_choose(prog, x, y, T, &mk, &chan, &v)) {
                    ok = true;
                    rec = make_spawn(key ^ mk, (int)cv.y, comp, chan, v, sg, phase ? -1 : 1, non, 1);
                }
            } else {
                int64_t sre, sim;
                const int64_t Pw = column_weight(prog, x, y, &sre, &sim);
                if (Pw >= (1ll << 52)) {
                    set_error(st, DERR_DT_TOO_LARGE);
                } else if (T < Pw) {
                    uint64_t mk;
                    int chan;
                    int64_t v;
                    ok = choose_destination(prog, x, y, sre, sim, T, &mk, &chan, &v);
                    if (ok) rec = make_spawn(key ^ mk, (int)cv.y, comp, chan, v, sg, phase ? -1 : 1, non, 1);
                    else set_error(st, DERR_TILE_CAPACITY);
                }
            }
        }
        const uint32_t bal = __ballot_sync(kFull, ok);
        const int nrec = __popc(bal);
        if (staged + nrec > kStage) {
            warp_flush(stage, staged, P, lane);
            staged = 0;
        }
        if (ok) stage[staged + __popc(bal & ((1u << lane) - 1u))] = rec;
        staged += nrec;
        __syncwarp();
    }
    if (staged) warp_flush(stage, staged, P, lane);
}

// ---------------------------------------------------------------------------
// Learned proposal (the library's extension; not in the paper).  A parent's
// attempting walker (T < p_att, as for the static proposal) draws its
// destination slot k from integer weights Q_k summing to 2^24 and each
// channel c of slot k receives floor(A) + Bernoulli(frac A) walkers with
// A = |c(L)| 2^24 / (Q_k p_att), so that the expected spawn is |c(L)| / 2^52
// per walker as in the plain method.  Q mixes the network's softmax over the
// column's destinations (share 1 - eps) with the static proposal (share eps):
//   L_k = floor((1 - eps) q_k 2^24),  S_k = floor(eps s_k / p_att 2^24),
//   Q_k = max(1, L_k + S_k) for s_k > 0 (else 0),
// the first largest Q_k absorbing 2^24 - sum Q.  The network runs in single
// precision with every operation rounded explicitly in a fixed order (no
// contraction), so that a CPU evaluating the same steps gets the same bits.
// ---------------------------------------------------------------------------

// e^x (x <= 0, else unused): 2^(x log2 e) = 2^k 2^f with k = floor, 2^f by
// the degree-7 Taylor polynomial of e^(f ln 2) in Horner form, 2^k placed in
// the exponent field.  Below -87 the result is 0.
__device__ __forceinline__ float lp_exp(float x)
{
    if (x < -87.0f) return 0.0f;
    const float y = __fmul_rn(x, 1.44269504f);
    const float k = floorf(y);
    const float f = __fsub_rn(y, k);
    float p = 1.52527338e-5f;   // (ln 2)^7 / 7!
    p = __fmaf_rn(p, f, 1.54035304e-4f);
    p = __fmaf_rn(p, f, 1.33335581e-3f);
    p = __fmaf_rn(p, f, 9.61812911e-3f);
    p = __fmaf_rn(p, f, 5.55041087e-2f);
    p = __fmaf_rn(p, f, 2.40226507e-1f);
    p = __fmaf_rn(p, f, 6.93147181e-1f);
    p = __fmaf_rn(p, f, 1.0f);
    return __fmul_rn(p, __int_as_float((int)(((uint32_t)((int)k + 127)) << 23)));
}

// Network layout in P.mlp: w1 [H x I], b1 [H], w2 [H x H], b2 [H], w3 [G x H], b3 [G].
struct LpNet {
    const float *w1, *b1, *w2, *b2, *w3, *b3;
    int I, H;
};

__device__ __forceinline__ LpNet lp_net(const StepParams& P)
{
    LpNet w;
    w.I = P.mlp_in;
    w.H = P.mlp_hidden;
    w.w1 = P.mlp;
    w.b1 = w.w1 + w.H * w.I;
    w.w2 = w.b1 + w.H;
    w.b2 = w.w2 + w.H * w.H;
    w.w3 = w.b2 + w.H;
    w.b3 = w.w3 + P.mlp_out * w.H;
    return w;
}

// First hidden layer, neuron j: b1 + the weights of the set input bits (x
// bits 0..n-1, then y bits), in ascending input order, then + w t by a fused
// multiply-add; ReLU.
__device__ __forceinline__ float lp_h1(const LpNet& w, int j, uint32_t x, uint32_t y, int n, float tf)
{
    const float* row = w.w1 + j * w.I;
    float a = __ldg(&w.b1[j]);
    for (int i = 0; i < n; ++i)
        if ((x >> i) & 1u) a = __fadd_rn(a, __ldg(&row[i]));
    for (int i = 0; i < n; ++i)
        if ((y >> i) & 1u) a = __fadd_rn(a, __ldg(&row[n + i]));
    a = __fmaf_rn(__ldg(&row[2 * n]), tf, a);
    return a > 0.0f ? a : 0.0f;
}

// Second hidden layer, neuron j: b2 then fused multiply-adds in ascending order; ReLU.
__device__ __forceinline__ float lp_h2(const LpNet& w, int j, const float* h1)
{
    const float* row = w.w2 + j * w.H;
    float a = __ldg(&w.b2[j]);
    for (int i = 0; i < w.H; ++i) a = __fmaf_rn(__ldg(&row[i]), h1[i], a);
    return a > 0.0f ? a : 0.0f;
}

// Logit of output g: b3 then fused multiply-adds in ascending order.
__device__ __forceinline__ float lp_logit(const LpNet& w, int g, const float* h2)
{
    const float* row = w.w3 + g * w.H;
    float a = __ldg(&w.b3[g]);
    for (int i = 0; i < w.H; ++i) a = __fmaf_rn(__ldg(&row[i]), h2[i], a);
    return a;
}

// Output index of a destination mask (masks sorted on the device), or -1.
__device__ __forceinline__ int lp_output(const StepParams& P, uint64_t mask)
{
    int lo = 0, hi = P.mlp_out;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (__ldg(&P.mlp_mask[mid]) < mask) lo = mid + 1; else hi = mid;
    }
    return (lo < P.mlp_out && __ldg(&P.mlp_mask[lo]) == mask) ? __ldg(&P.mlp_idx[lo]) : -1;
}

// Static weight of slot k.
__device__ __forceinline__ int64_t slot_width(const Prog& prog, int k)
{
    return prog.stat[k].end - (k ? prog.stat[k - 1].end : 0);
}

// Q_k from the slot's exponential e (valid when has_out) and the softmax sum S.
__device__ __forceinline__ int64_t lp_q(float e, bool has_out, float S, float eps, int64_t width, int64_t p_att)
{
    if (width <= 0) return 0;
    int64_t L = 0;
    if (has_out && S > 0.0f) {
        const float q = __fdiv_rn(e, S);
        L = (int64_t)floorf(__fmul_rn(__fmul_rn(__fsub_rn(1.0f, eps), q), 16777216.0f));
    }
    const int64_t St = (int64_t)floor(__dmul_rn(__ddiv_rn(__dmul_rn((double)eps, (double)width), (double)p_att),
                                                16777216.0));
    const int64_t Q = L + St;
    return Q < 1 ? 1 : Q;
}

// The walker's randomness: two Philox calls keyed like its spawn draw with the
// learned kind; V (24 bits) picks the slot, u_re and u_im (53 bits each) the
// Bernoulli parts of the two channels.
__device__ __forceinline__ void lp_draws(uint64_t key, int phase, int comp, uint32_t j, uint2 kd, uint32_t* V,
                                         double* ure, double* uim)
{
    uint4 c = make_uint4((uint32_t)key, (uint32_t)(key >> 32), (uint32_t)phase | ((uint32_t)comp << 1) | (kKindLearned << 2),
                         ((j >> 1) << 2) | ((j & 1u) << 1));
    const uint4 a = philox10(c, kd);
    c.w |= 1u;
    const uint4 b = philox10(c, kd);
    *V = a.x >> 8;
    *ure = __dmul_rn((double)((((uint64_t)a.y) << 21) | (a.z >> 11)), 1.0 / 9007199254740992.0);
    *uim = __dmul_rn((double)((((uint64_t)b.x) << 21) | (b.y >> 11)), 1.0 / 9007199254740992.0);
}

// Walkers on channel value v of a slot with proposal weight Q: floor(A) +
// (u < frac A), A = |v| 2^24 / (Q p_att).
__device__ __forceinline__ int64_t lp_count(int64_t v, int64_t Q, int64_t p_att, double u)
{
    const int64_t w = iabs64(v);
    if (w == 0) return 0;
    const double A = __ddiv_rn(__dmul_rn((double)w, 16777216.0), __dmul_rn((double)Q, (double)p_att));
    const double fl = floor(A);
    return (int64_t)fl + (u < __dsub_rn(A, fl) ? 1 : 0);
}

// Light parents under the learned proposal: one thread per candidate (an
// attempting walker); the network is evaluated for the candidate's source,
// and up to two records (Re, Im channel of the drawn destination) are staged.
__global__ void __launch_bounds__(kThreads, 2) k_spawn_learned(StepParams P)
{
    __shared__ __align__(16) uint8_t sprog[2][kProgSmem];
    __shared__ __align__(16) SRec sstage[kThreads / 32][kStage];
    DevState* st = P.st;
    if (cta_error(st)) return;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const StepInfo inf = P.info[st->call_index];
    const int cur = st->cur, prv = (cur + 2) % 3;
    const Rec* src0 = P.pop[cur];
    const Rec* src1 = P.pop[prv];
    // one instance (the learned proposal takes no batch): both programs staged
    const uint8_t* pb0 = stage_prog(prog_ptr(P, inf, 0, 0), sprog[0]);
    const uint8_t* pb1 = stage_prog(prog_ptr(P, inf, 0, inf.ab2 ? 1 : 0), sprog[1]);
    __syncthreads();
    const LpNet net = lp_net(P);
    const int64_t total = min(st->cand_total, P.cand_cap);
    SRec* stage = sstage[warp];
    int staged = 0;
    const int64_t stride = (int64_t)gridDim.x * kThreads;
    for (int64_t base = (int64_t)blockIdx.x * kThreads + warp * 32; base < total; base += stride) {
        const int64_t i = base + lane;
        SRec rec[2];
        bool ok[2] = {false, false};
        if (i < total) {
            const uint4 cv = __ldcs((const uint4*)P.cand + i);
            const int comp = (int)((cv.w >> 20) & 1u), phase = (int)((cv.w >> 21) & 1u);
            const int non = (int)((cv.w >> 22) & 1u), sg = ((cv.w >> 23) & 1u) ? 1 : -1;
            const uint32_t j = cv.w & kJ20;
            const uint32_t rank = cv.x - (uint32_t)__ldg(&P.segoff[phase ? prv : cur][cv.y]);
            const int64_t T = walker_T(cv.z, rank, j, comp, phase, P.kd[cv.y]);
            const uint64_t key = __ldg(&(phase ? src1 : src0)[cv.x].key);
            const int n = P.seginfo[cv.y].n;
            const uint32_t x = (uint32_t)(key >> n), y = (uint32_t)(key & (n == 32 ? 0xFFFFFFFFu : ((1u << n) - 1u)));
            const Prog prog = prog_at(phase ? pb1 : pb0);
            const int64_t p_att = prog.h->p_att;
            const int ns = prog.h->n_stat;
            if (p_att >= (1ll << 52)) {
                set_error(st, DERR_DT_TOO_LARGE);
            } else if (T < p_att) {   // an attempting walker
                const float tf32 = __double2float_rn(inf.t[phase]);
                float h1[kMaxHidden], h2[kMaxHidden];
                for (int q = 0; q < net.H; ++q) h1[q] = lp_h1(net, q, x, y, n, tf32);
                for (int q = 0; q < net.H; ++q) h2[q] = lp_h2(net, q, h1);
                // e[k]: logit, then its exponential; g[k] >= 0 where the slot has an output
                float e[kMaxLearnedSlots];
                int16_t g[kMaxLearnedSlots];
                float m = -INFINITY;
                for (int k = 0; k < ns; ++k) {
                    g[k] = (int16_t)(slot_width(prog, k) > 0 ? lp_output(P, prog.stat[k].mask) : -1);
                    if (g[k] >= 0) {
                        e[k] = lp_logit(net, g[k], h2);
                        if (e[k] > m) m = e[k];
                    }
                }
                float S = 0.0f;
                for (int k = 0; k < ns; ++k)
                    if (g[k] >= 0) {
                        e[k] = lp_exp(__fsub_rn(e[k], m));
                        S = __fadd_rn(S, e[k]);
                    }
                int64_t sum = 0, qa = -1;
                int arg = -1;
                for (int k = 0; k < ns; ++k) {
                    const int64_t w = slot_width(prog, k);
                    if (w <= 0) continue;
                    const int64_t Q = lp_q(e[k], g[k] >= 0, S, P.mlp_eps, w, p_att);
                    sum += Q;
                    if (arg < 0 || Q > qa) {
                        arg = k;
                        qa = Q;
                    }
                }
                uint32_t V;
                double u[2];
                lp_draws(key, phase, comp, j, P.kd[cv.y], &V, &u[0], &u[1]);
                int64_t cum = 0, Qk = 0;
                int k = 0;
                for (; k < ns; ++k) {
                    const int64_t w = slot_width(prog, k);
                    Qk = w <= 0 ? 0 : lp_q(e[k], g[k] >= 0, S, P.mlp_eps, w, p_att);
                    if (k == arg) Qk += (1ll << 24) - sum;
                    cum += Qk;
                    if ((int64_t)V < cum) break;
                }
                if (k < ns) {
                    int64_t v[2];
                    value_at_mask(prog, prog.stat[k].mask, x, y, &v[0], &v[1]);
                    for (int c = 0; c < 2; ++c) {
                        const int64_t cnt = lp_count(v[c], Qk, p_att, u[c]);
                        if (cnt == 0) continue;
                        if (cnt > 0x7FFFFFFFll) {
                            set_error(st, DERR_POP_OVERFLOW);
                            continue;
                        }
                        ok[c] = true;
                        rec[c] = make_spawn(key ^ prog.stat[k].mask, (int)cv.y, comp, c, v[c], sg, phase ? -1 : 1, non,
                                            (int32_t)cnt);
                    }
                }
            }
        }
#pragma unroll
        for (int c = 0; c < 2; ++c) {
            const uint32_t bal = __ballot_sync(kFull, ok[c]);
            const int nrec = __popc(bal);
            if (staged + nrec > kStage) {
                warp_flush(stage, staged, P, lane);
                staged = 0;
            }
            if (ok[c]) stage[staged + __popc(bal & ((1u << lane) - 1u))] = rec[c];
            staged += nrec;
            __syncwarp();
        }
    }
    if (staged) warp_flush(stage, staged, P, lane);
}

// ---------------------------------------------------------------------------
// Learned proposal on the tensor cores (QMC_PROPOSAL_LEARNED_TC; the
// library's extension, not in the paper).  The same proposal as above --
// integer weights Q_k summing to 2^24 from the network's softmax (share
// 1 - eps) and the static proposal (share eps), floor + Bernoulli walker
// counts -- with the network evaluated as bf16 matrix products with fp32
// accumulation (mma.sync m16n8k16) and GELU activations: one warp evaluates
// 16 sources at once, hidden activations stay in registers between layers.
// Unbiased for any Q (Q_k >= 1 wherever the column can be nonzero), so the
// rounding of the products changes the variance only, never the mean; the
// products of a source do not depend on the other rows of its tile, so a
// parent gets the same Q on the light and the heavy path.
// ---------------------------------------------------------------------------
constexpr int kTcWarps = 4;                       // warps per CTA of the light kernel
constexpr int kTcMaxH = 64, kTcMaxGp = 256, kTcMaxIp = 80;

// Input c of a source: bit c of x, bit c - n of y, then t; 0 past the inputs.
__device__ __forceinline__ float tc_feat(uint32_t x, uint32_t y, float t, int c, int n)
{
    return c < n ? (float)((x >> c) & 1u) : (c < 2 * n ? (float)((y >> (c - n)) & 1u) : (c == 2 * n ? t : 0.0f));
}

// Logits of 16 sources by one warp.  The lane's fragment rows are g = lane /
// 4 (source a: xa, ya, ta) and g + 8 (source b); the weights are in shared
// memory in the TcLayout; logits go to out[row * ldo + output] (fp32, all Gp
// outputs).
__device__ void tc_forward(const uint8_t* sw, const TcLayout& L, int n, uint32_t xa, uint32_t ya, float ta,
                           uint32_t xb, uint32_t yb, float tb, float* out, int ldo, int lane)
{
    const int g = lane >> 2, tig = lane & 3;
    const __nv_bfloat16* W1 = (const __nv_bfloat16*)(sw + L.o_w1);
    const __nv_bfloat16* W2 = (const __nv_bfloat16*)(sw + L.o_w2);
    const __nv_bfloat16* W3 = (const __nv_bfloat16*)(sw + L.o_w3);
    const float* b1 = (const float*)(sw + L.o_b1);
    const float* b2 = (const float*)(sw + L.o_b2);
    const float* b3 = (const float*)(sw + L.o_b3);
    const int nth = L.H / 8, kth = L.H / 16, kt1 = L.Ip / 16;
    float acc[kTcMaxH / 8][4];
    uint32_t a[kTcMaxH / 16][4];
    // layer 1
#pragma unroll
    for (int nt = 0; nt < kTcMaxH / 8; ++nt) {
        const int c = nt * 8 + 2 * tig;
        acc[nt][0] = nt < nth ? b1[c] : 0.0f;
        acc[nt][1] = nt < nth ? b1[c + 1] : 0.0f;
        acc[nt][2] = acc[nt][0];
        acc[nt][3] = acc[nt][1];
    }
#pragma unroll
    for (int kt = 0; kt < kTcMaxIp / 16; ++kt) {
        if (kt >= kt1) break;
        const int c = kt * 16 + 2 * tig;
        uint32_t f[4];
        f[0] = bf16x2(tc_feat(xa, ya, ta, c, n), tc_feat(xa, ya, ta, c + 1, n));
        f[1] = bf16x2(tc_feat(xb, yb, tb, c, n), tc_feat(xb, yb, tb, c + 1, n));
        f[2] = bf16x2(tc_feat(xa, ya, ta, c + 8, n), tc_feat(xa, ya, ta, c + 9, n));
        f[3] = bf16x2(tc_feat(xb, yb, tb, c + 8, n), tc_feat(xb, yb, tb, c + 9, n));
#pragma unroll
        for (int nt = 0; nt < kTcMaxH / 8; ++nt) {
            if (nt >= nth) break;
            const uint32_t* row = (const uint32_t*)(W1 + (nt * 8 + g) * L.ld1 + kt * 16 + 2 * tig);
            mma_bf16(acc[nt], f, row[0], row[4]);
        }
    }
    // GELU, repacked as the next layer's A fragments (two 8-column tiles per 16-column k tile)
#pragma unroll
    for (int kt = 0; kt < kTcMaxH / 16; ++kt) {
        a[kt][0] = bf16x2(tc_gelu(acc[2 * kt][0]), tc_gelu(acc[2 * kt][1]));
        a[kt][1] = bf16x2(tc_gelu(acc[2 * kt][2]), tc_gelu(acc[2 * kt][3]));
        a[kt][2] = bf16x2(tc_gelu(acc[2 * kt + 1][0]), tc_gelu(acc[2 * kt + 1][1]));
        a[kt][3] = bf16x2(tc_gelu(acc[2 * kt + 1][2]), tc_gelu(acc[2 * kt + 1][3]));
    }
    // layer 2
#pragma unroll
    for (int nt = 0; nt < kTcMaxH / 8; ++nt) {
        const int c = nt * 8 + 2 * tig;
        acc[nt][0] = nt < nth ? b2[c] : 0.0f;
        acc[nt][1] = nt < nth ? b2[c + 1] : 0.0f;
        acc[nt][2] = acc[nt][0];
        acc[nt][3] = acc[nt][1];
    }
#pragma unroll
    for (int kt = 0; kt < kTcMaxH / 16; ++kt) {
        if (kt >= kth) break;
#pragma unroll
        for (int nt = 0; nt < kTcMaxH / 8; ++nt) {
            if (nt >= nth) break;
            const uint32_t* row = (const uint32_t*)(W2 + (nt * 8 + g) * L.ld2 + kt * 16 + 2 * tig);
            mma_bf16(acc[nt], a[kt], row[0], row[4]);
        }
    }
#pragma unroll
    for (int kt = 0; kt < kTcMaxH / 16; ++kt) {
        a[kt][0] = bf16x2(tc_gelu(acc[2 * kt][0]), tc_gelu(acc[2 * kt][1]));
        a[kt][1] = bf16x2(tc_gelu(acc[2 * kt][2]), tc_gelu(acc[2 * kt][3]));
        a[kt][2] = bf16x2(tc_gelu(acc[2 * kt + 1][0]), tc_gelu(acc[2 * kt + 1][1]));
        a[kt][3] = bf16x2(tc_gelu(acc[2 * kt + 1][2]), tc_gelu(acc[2 * kt + 1][3]));
    }
    // layer 3: one 8-output tile at a time, straight to shared memory
    for (int nt = 0; nt < L.Gp / 8; ++nt) {
        const int c = nt * 8 + 2 * tig;
        float d[4] = {b3[c], b3[c + 1], b3[c], b3[c + 1]};
#pragma unroll
        for (int kt = 0; kt < kTcMaxH / 16; ++kt) {
            if (kt >= kth) break;
            const uint32_t* row = (const uint32_t*)(W3 + (nt * 8 + g) * L.ld3 + kt * 16 + 2 * tig);
            mma_bf16(d, a[kt], row[0], row[4]);
        }
        out[g * ldo + c] = d[0];
        out[g * ldo + c + 1] = d[1];
        out[(g + 8) * ldo + c] = d[2];
        out[(g + 8) * ldo + c + 1] = d[3];
    }
}

// Per program (pass): each static slot's network output (-1: none; -2: the
// slot has width 0 and is never chosen) and its static part S_k = floor(eps
// s_k / p_att 2^24) (< 2^24).
struct TcSlots {
    int16_t out[kMaxLearnedSlots];
    int32_t st[kMaxLearnedSlots];
};

__device__ void tc_slots_fill(const StepParams& P, const Prog& prog, TcSlots* s, int tid, int nthr)
{
    const int64_t p_att = prog.h->p_att;
    for (int k = tid; k < prog.h->n_stat; k += nthr) {
        const int64_t w = slot_width(prog, k);
        s->out[k] = (int16_t)(w > 0 ? lp_output(P, prog.stat[k].mask) : -2);
        s->st[k] = (w > 0 && p_att > 0 && p_att < (1ll << 52))
                       ? (int32_t)floor(__dmul_rn(__ddiv_rn(__dmul_rn((double)P.mlp_eps, (double)w), (double)p_att),
                                                  16777216.0))
                       : 0;
    }
}

// The weights Q_k of one source from its logits lg (by output; overwritten
// with the exponentials by tc_row_prepare): m = max over the slots with an
// output, e = exp(z - m), S = (sum of e over the even slots, in order) + (the
// same over the odd slots), c = (1 - eps) 2^24 / S,
// L_k = floor(e_k c), Q_k = max(1, L_k + S_k) on slots of positive width, the
// first largest absorbing 2^24 - sum Q.  One thread per source; the light and
// the heavy kernels share these functions, so a parent's Q is the same on
// either path.
struct TcRow {
    float c;
    int arg;
    int64_t rem;
};

__device__ __forceinline__ int64_t tc_q(const float* lg, const TcSlots* s, int k, float c)
{
    const int o = s->out[k];
    const int64_t L = o >= 0 ? (int64_t)floorf(__fmul_rn(lg[o], c)) : 0;
    const int64_t Q = L + s->st[k];
    return Q < 1 ? 1 : Q;
}

__device__ TcRow tc_row_prepare(float* lg, const TcSlots* s, int ns, float eps)
{
    float m = -INFINITY;
    for (int k = 0; k < ns; ++k)
        if (s->out[k] >= 0) m = fmaxf(m, lg[s->out[k]]);
    float Sh[2] = {0.0f, 0.0f};
    for (int k = 0; k < ns; ++k) {
        const int o = s->out[k];
        if (o < 0) continue;
        const float e = expf(__fsub_rn(lg[o], m));
        lg[o] = e;
        Sh[k & 1] = __fadd_rn(Sh[k & 1], e);
    }
    const float S = __fadd_rn(Sh[0], Sh[1]);
    TcRow r;
    r.c = S > 0.0f ? __fdiv_rn(__fmul_rn(__fsub_rn(1.0f, eps), 16777216.0f), S) : 0.0f;
    int64_t sum = 0, qa = -1;
    int arg = -1;
    for (int k = 0; k < ns; ++k) {
        if (s->out[k] == -2) continue;
        const int64_t Q = tc_q(lg, s, k, r.c);
        sum += Q;
        if (Q > qa) {
            qa = Q;
            arg = k;
        }
    }
    r.arg = arg;
    r.rem = (1ll << 24) - sum;
    return r;
}

// The slot whose interval [cum_{k-1}, cum_k) of the weights holds V (ns when
// none does) and its weight *Qk.
__device__ int tc_row_choose(const float* lg, const TcSlots* s, int ns, const TcRow& r, uint32_t V, int64_t* Qk)
{
    int64_t cum = 0;
    for (int k = 0; k < ns; ++k) {
        if (s->out[k] == -2) continue;
        const int64_t Q = tc_q(lg, s, k, r.c) + (k == r.arg ? r.rem : 0);
        cum += Q;
        if ((int64_t)V < cum) {
            *Qk = Q;
            return k;
        }
    }
    *Qk = 0;
    return ns;
}

// The same weights and choice for the rows of a 16-row logit tile, two lanes
// per row (lane r and lane r + 16 take the even and the odd slots of row
// r = lane & 15): the max and the integer sums do not depend on the order,
// and the float sum is the even slots' sum plus the odd slots', as in
// tc_row_prepare.  Every lane runs the same number of iterations (nsmax, the
// larger slot count of the two passes); act = the row is in use.
__device__ TcRow tc_pair_prepare(float* lg, const TcSlots* s, int ns, int nsmax, float eps, bool act, int half)
{
    float m = -INFINITY;
    for (int k = half; k < nsmax; k += 2)
        if (act && k < ns && s->out[k] >= 0) m = fmaxf(m, lg[s->out[k]]);
    m = fmaxf(m, __shfl_xor_sync(kFull, m, 16));
    float S = 0.0f;
    for (int k = half; k < nsmax; k += 2) {
        if (!act || k >= ns) continue;
        const int o = s->out[k];
        if (o < 0) continue;
        const float e = expf(__fsub_rn(lg[o], m));
        lg[o] = e;
        S = __fadd_rn(S, e);
    }
    const float So = __shfl_xor_sync(kFull, S, 16);
    const float St = half ? __fadd_rn(So, S) : __fadd_rn(S, So);
    TcRow r;
    r.c = St > 0.0f ? __fdiv_rn(__fmul_rn(__fsub_rn(1.0f, eps), 16777216.0f), St) : 0.0f;
    int64_t sum = 0, qa = -1;
    int arg = -1;
    for (int k = half; k < nsmax; k += 2) {
        if (!act || k >= ns || s->out[k] == -2) continue;
        const int64_t Q = tc_q(lg, s, k, r.c);
        sum += Q;
        if (Q > qa) {
            qa = Q;
            arg = k;
        }
    }
    sum += __shfl_xor_sync(kFull, sum, 16);
    const int64_t qo = __shfl_xor_sync(kFull, qa, 16);
    const int ao = __shfl_xor_sync(kFull, arg, 16);
    if (qo > qa || (qo == qa && ao >= 0 && (arg < 0 || ao < arg))) {
        qa = qo;
        arg = ao;
    }
    r.arg = arg;
    r.rem = (1ll << 24) - sum;
    return r;
}

__device__ int tc_pair_choose(const float* lg, const TcSlots* s, int ns, int nsmax, const TcRow& r, uint32_t V,
                              bool act, int half, int64_t* Qk)
{
    int64_t cum = 0, qf = 0;
    int found = act ? -1 : ns;
    for (int i = 0; 2 * i < nsmax; ++i) {
        const int k = 2 * i + half;
        int64_t q = 0;
        if (found < 0 && k < ns && s->out[k] != -2) q = tc_q(lg, s, k, r.c) + (k == r.arg ? r.rem : 0);
        const int64_t qp = __shfl_xor_sync(kFull, q, 16);
        const int64_t qe = half ? qp : q, qd = half ? q : qp;
        if (found < 0) {
            if ((int64_t)V < cum + qe) {
                found = 2 * i;
                qf = qe;
            } else if ((int64_t)V < cum + qe + qd) {
                found = 2 * i + 1;
                qf = qd;
            } else {
                cum += qe + qd;
            }
        }
        if (__all_sync(kFull, found >= 0)) break;
    }
    if (found < 0 || found >= ns) {
        *Qk = 0;
        return ns;
    }
    *Qk = qf;
    return found;
}

// Light parents under the tensor-core proposal: each warp takes 16
// candidates at a time.  Shared memory: the network (TcLayout), the slot
// tables of both passes, one 16-row logit tile per warp.
__global__ void __launch_bounds__(kTcWarps * 32) k_spawn_learned_tc(StepParams P)
{
    extern __shared__ __align__(16) uint8_t tsm[];
    __shared__ __align__(16) SRec sstage[kTcWarps][kStage];
    DevState* st = P.st;
    if (cta_error(st)) return;
    const TcLayout L = tc_layout(P.mlp_in, P.mlp_hidden, P.mlp_out);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nthr = kTcWarps * 32;
    for (int i = threadIdx.x; i < L.bytes / 16; i += nthr) ((uint4*)tsm)[i] = ((const uint4*)P.mlp_tc)[i];
    TcSlots* slots = (TcSlots*)(tsm + L.bytes);
    const int ldo = L.Gp + 4;
    float* lgt = (float*)(tsm + L.bytes + 2 * sizeof(TcSlots)) + warp * 16 * ldo;
    const StepInfo inf = P.info[st->call_index];
    const int cur = st->cur, prv = (cur + 2) % 3;
    const Prog prog[2] = {prog_at(prog_ptr(P, inf, 0, 0)), prog_at(prog_ptr(P, inf, 0, inf.ab2 ? 1 : 0))};
    for (int ph = 0; ph < 2; ++ph) tc_slots_fill(P, prog[ph], slots + ph, threadIdx.x, nthr);
    __syncthreads();
    const int64_t total = min(st->cand_total, P.cand_cap);
    SRec* stage = sstage[warp];
    int staged = 0;
    const int n = P.seginfo[0].n;
    const uint32_t ymask = n == 32 ? 0xFFFFFFFFu : ((1u << n) - 1u);
    const float tph[2] = {__double2float_rn(inf.t[0]), __double2float_rn(inf.t[1])};
    const int64_t ntiles = (total + 15) / 16;
    for (int64_t tile = (int64_t)blockIdx.x * kTcWarps + warp; tile < ntiles; tile += (int64_t)gridDim.x * kTcWarps) {
        const int64_t i = tile * 16 + lane;
        // lanes 0..15: one candidate each
        bool att = false;
        uint32_t x = 0u, y = 0u, j = 0u, seg = 0u;
        int comp = 0, phase = 0, non = 0, sg = 1;
        uint64_t key = 0ull;
        if (lane < 16 && i < total) {
            const uint4 cv = __ldcs((const uint4*)P.cand + i);
            comp = (int)((cv.w >> 20) & 1u);
            phase = (int)((cv.w >> 21) & 1u);
            non = (int)((cv.w >> 22) & 1u);
            sg = ((cv.w >> 23) & 1u) ? 1 : -1;
            j = cv.w & kJ20;
            seg = cv.y;
            const uint32_t rank = cv.x - (uint32_t)__ldg(&P.segoff[phase ? prv : cur][cv.y]);
            const int64_t T = walker_T(cv.z, rank, j, comp, phase, P.kd[cv.y]);
            const int64_t p_att = prog[phase].h->p_att;
            if (p_att >= (1ll << 52)) set_error(st, DERR_DT_TOO_LARGE);
            att = p_att < (1ll << 52) && T < p_att;
            key = __ldg(&(phase ? P.pop[prv] : P.pop[cur])[cv.x].key);
            x = (uint32_t)(key >> n);
            y = (uint32_t)(key & ymask);
        }
        const int ga = lane >> 2, gb = ga + 8;
        const uint32_t xa = __shfl_sync(kFull, x, ga), ya = __shfl_sync(kFull, y, ga);
        const uint32_t xb = __shfl_sync(kFull, x, gb), yb = __shfl_sync(kFull, y, gb);
        const float ta = tph[__shfl_sync(kFull, phase, ga)], tb = tph[__shfl_sync(kFull, phase, gb)];
        tc_forward(tsm, L, n, xa, ya, __bfloat162float(__float2bfloat16_rn(ta)), xb, yb,
                   __bfloat162float(__float2bfloat16_rn(tb)), lgt, ldo, lane);
        __syncwarp();
        SRec rec[2];
        bool ok[2] = {false, false};
        // the rows' weights and choices, two lanes per row
        uint32_t V = 0u;
        double u[2] = {0.0, 0.0};
        if (att) lp_draws(key, phase, comp, j, P.kd[seg], &V, &u[0], &u[1]);
        const int r = lane & 15, half = lane >> 4;
        const bool ract = __shfl_sync(kFull, att, r);
        const int rph = __shfl_sync(kFull, phase, r);
        const uint32_t rV = __shfl_sync(kFull, V, r);
        const int rns = prog[rph].h->n_stat;
        const int nsmax = max(prog[0].h->n_stat, prog[1].h->n_stat);
        float* rlg = lgt + r * ldo;
        const TcRow tr = tc_pair_prepare(rlg, slots + rph, rns, nsmax, P.mlp_eps, ract, half);
        int64_t Qk;
        const int k = tc_pair_choose(rlg, slots + rph, rns, nsmax, tr, rV, ract, half, &Qk);
        if (att) {
            const Prog& pg = prog[phase];
            if (k < pg.h->n_stat) {
                int64_t v[2];
                value_at_mask(pg, pg.stat[k].mask, x, y, &v[0], &v[1]);
                for (int c = 0; c < 2; ++c) {
                    const int64_t cnt = lp_count(v[c], Qk, pg.h->p_att, u[c]);
                    if (cnt == 0) continue;
                    if (cnt > 0x7FFFFFFFll) {
                        set_error(st, DERR_POP_OVERFLOW);
                        continue;
                    }
                    ok[c] = true;
                    rec[c] = make_spawn(key ^ pg.stat[k].mask, (int)seg, comp, c, v[c], sg, phase ? -1 : 1, non,
                                        (int32_t)cnt);
                }
            }
        }
#pragma unroll
        for (int c = 0; c < 2; ++c) {
            const uint32_t bal = __ballot_sync(kFull, ok[c]);
            const int nrec = __popc(bal);
            if (staged + nrec > kStage) {
                warp_flush(stage, staged, P, lane);
                staged = 0;
            }
            if (ok[c]) stage[staged + __popc(bal & ((1u << lane) - 1u))] = rec[c];
            staged += nrec;
            __syncwarp();
        }
    }
    if (staged) warp_flush(stage, staged, P, lane);
}

__host__ __device__ __forceinline__ int tc_smem_bytes(const TcLayout& L, int warps)
{
    return L.bytes + 2 * (int)sizeof(TcSlots) + warps * 16 * (L.Gp + 4) * 4;
}

// ---------------------------------------------------------------------------
// Spawning, heavy parents: one CTA per chunk of kHeavyChunk walkers of one
// parent component.  The column is evaluated once into shared memory as a
// cumulative weight table; each spawned walker finds its interval from a
// table of the first bin of every 2^s-wide slice of [0, P) (at most 1024
// slices) and a short forward scan, usually one or two cumulative weights;
// counts are aggregated per (destination, channel) and emitted as one record
// each.
// ---------------------------------------------------------------------------
template <bool kLearned, bool kTc>
__device__ __forceinline__ void spawn_heavy(const StepParams& P)
{
    __shared__ int64_t cum[2 * kMaxEntries];
    __shared__ int64_t vals[2 * kMaxEntries];
    __shared__ __align__(8) int hist[2 * kMaxEntries];
    __shared__ int64_t warp_tot[kThreads / 32];
    __shared__ float s_h1[kMaxHidden], s_h2[kMaxHidden], s_e[kMaxLearnedSlots];
    __shared__ int16_t s_g[kMaxLearnedSlots];
    __shared__ float s_S;
    __shared__ unsigned long long s_base;
    __shared__ int s_nout;
    __shared__ uint16_t sidx[1025];   // first bin of each 2^ish-wide slice of [0, Pw)
    __shared__ int64_t s_col[3];      // P, Re and Im of the diagonal element of the parent's column
    DevState* st = P.st;
    if (cta_error(st)) return;
    const int64_t nitems = min(st->heavy_total, P.heavy_cap);
    if (nitems == 0) return;
    const int ci = st->call_index;
    const StepInfo inf = P.info[ci];
    const int cur = st->cur, prv = (cur + 2) % 3;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    // learned proposal: 64-bit walker counts per (slot, channel) bin, over hist
    unsigned long long* lh = (unsigned long long*)hist;
    // tensor-core proposal: the network, one program's slot table and a 16-row logit tile (dynamic)
    extern __shared__ __align__(16) uint8_t hsm[];
    const TcLayout TL = tc_layout(P.mlp_in, P.mlp_hidden, P.mlp_out);
    TcSlots* hslots = (TcSlots*)(hsm + TL.bytes);
    const int hldo = TL.Gp + 4;
    float* hlg = (float*)(hsm + TL.bytes + sizeof(TcSlots));
    if (kTc) {
        for (int i = tid; i < TL.bytes / 16; i += kThreads) ((uint4*)hsm)[i] = ((const uint4*)P.mlp_tc)[i];
        __syncthreads();
    }

    for (int64_t item = blockIdx.x; item < nitems; item += gridDim.x) {
        const HeavyItem it = P.heavy[item];
        const SegInfo si = P.seginfo[it.seg];
        const int n = si.n;
        const uint32_t ymask = n == 32 ? 0xFFFFFFFFu : ((1u << n) - 1u);
        const Prog prog = prog_at(prog_ptr(P, inf, si.inst, it.phase));
        const Rec par = (it.phase ? P.pop[prv] : P.pop[cur])[it.parent];
        const uint32_t x = (uint32_t)(par.key >> n), y = (uint32_t)(par.key & ymask);
        // bins of the walkers' draw T: plain, two per destination entry (Re,
        // Im; widths |Re L|, |Im L| over [0, P)); static proposal, three per
        // static slot (Re, Im and the rest of the slot's static weight, which
        // spawns nothing; over [0, p_att)); learned proposal, two per slot
        // (walker counts; the slot comes from the weights Q, not from T)
        const bool prop = P.proposal == 1, learned = kLearned;
        int64_t Pw;
        int nb;
        if (prop || learned) {
            Pw = prog.h->p_att;
            nb = (learned ? 2 : 3) * prog.h->n_stat;
        } else {
            // the column's weight and diagonal element, once per chunk
            if (tid == 0) {
                int64_t a, b;
                s_col[0] = column_weight(prog, x, y, &a, &b);
                s_col[1] = a;
                s_col[2] = b;
            }
            __syncthreads();
            Pw = s_col[0];
            const int64_t sre = s_col[1], sim = s_col[2];
            nb = 2 * prog.h->n_entry;
            if (nb <= 2 * kMaxEntries)
                for (int e = tid; e < prog.h->n_entry; e += kThreads) {
                    int64_t vr, vi;
                    entry_value(prog, prog.ent[e], x, y, sre, sim, &vr, &vi);
                    vals[2 * e] = vr;
                    vals[2 * e + 1] = vi;
                }
        }
        if (Pw >= (1ll << 52)) {
            if (threadIdx.x == 0) set_error(st, DERR_DT_TOO_LARGE);
            return;
        }
        if (nb > 2 * kMaxEntries || (learned && prog.h->n_stat > kMaxLearnedSlots)) {
            if (tid == 0) set_error(st, DERR_TILE_CAPACITY);
            return;
        }
        if (prop)
            for (int k = tid; k < prog.h->n_stat; k += kThreads) {
                int64_t vr, vi;
                value_at_mask(prog, prog.stat[k].mask, x, y, &vr, &vi);
                const int64_t width = slot_width(prog, k);
                vals[3 * k] = vr;
                vals[3 * k + 1] = vi;
                vals[3 * k + 2] = width - iabs64(vr) - iabs64(vi);   // no-spawn remainder
            }
        const int ns = prog.h->n_stat;
        if (learned && kTc) {
            // the source's weights Q (cum[k], then their inclusive prefix), the
            // network on the tensor cores as on the light path (every row of the tile the parent)
            for (int k = tid; k < ns; k += kThreads) {
                int64_t vr, vi;
                value_at_mask(prog, prog.stat[k].mask, x, y, &vr, &vi);
                vals[2 * k] = vr;
                vals[2 * k + 1] = vi;
            }
            for (int b = tid; b < nb; b += kThreads) lh[b] = 0ull;
            tc_slots_fill(P, prog, hslots, tid, kThreads);
            if (warp == 0) {
                const float tb = __bfloat162float(__float2bfloat16_rn(__double2float_rn(inf.t[it.phase])));
                tc_forward(hsm, TL, n, x, y, tb, x, y, tb, hlg, hldo, lane);
            }
            __syncthreads();
            if (tid == 0) {
                const TcRow r = tc_row_prepare(hlg, hslots, ns, P.mlp_eps);
                int64_t run = 0;
                for (int k = 0; k < ns; ++k) {
                    if (hslots->out[k] != -2) run += tc_q(hlg, hslots, k, r.c) + (k == r.arg ? r.rem : 0);
                    cum[k] = run;
                }
            }
            __syncthreads();
        } else if (learned) {
            // the source's weights Q (cum[k], then their inclusive prefix)
            const LpNet net = lp_net(P);
            const float tf32 = __double2float_rn(inf.t[it.phase]);
            for (int k = tid; k < ns; k += kThreads) {
                int64_t vr, vi;
                value_at_mask(prog, prog.stat[k].mask, x, y, &vr, &vi);
                vals[2 * k] = vr;
                vals[2 * k + 1] = vi;
            }
            for (int b = tid; b < nb; b += kThreads) lh[b] = 0ull;
            if (tid < net.H) s_h1[tid] = lp_h1(net, tid, x, y, n, tf32);
            __syncthreads();
            if (tid < net.H) s_h2[tid] = lp_h2(net, tid, s_h1);
            __syncthreads();
            for (int k = tid; k < ns; k += kThreads) {
                const int g = slot_width(prog, k) > 0 ? lp_output(P, prog.stat[k].mask) : -1;
                s_g[k] = (int16_t)g;
                if (g >= 0) s_e[k] = lp_logit(net, g, s_h2);
            }
            __syncthreads();
            if (tid == 0) {
                float m = -INFINITY;
                for (int k = 0; k < ns; ++k)
                    if (s_g[k] >= 0 && s_e[k] > m) m = s_e[k];
                float S = 0.0f;
                for (int k = 0; k < ns; ++k)
                    if (s_g[k] >= 0) {
                        s_e[k] = lp_exp(__fsub_rn(s_e[k], m));
                        S = __fadd_rn(S, s_e[k]);
                    }
                s_S = S;
            }
            __syncthreads();
            for (int k = tid; k < ns; k += kThreads)
                cum[k] = lp_q(s_e[k], s_g[k] >= 0, s_S, P.mlp_eps, slot_width(prog, k), Pw);
            __syncthreads();
            if (tid == 0) {
                int64_t sum = 0;
                int arg = -1;
                for (int k = 0; k < ns; ++k) {
                    if (slot_width(prog, k) <= 0) continue;
                    sum += cum[k];
                    if (arg < 0 || cum[k] > cum[arg]) arg = k;
                }
                if (arg >= 0) cum[arg] += (1ll << 24) - sum;
                for (int k = 1; k < ns; ++k) cum[k] += cum[k - 1];
            }
            __syncthreads();
        } else {
            for (int b = tid; b < nb; b += kThreads) hist[b] = 0;
            __syncthreads();
            // inclusive prefix of the bin widths (blocked per thread, then across threads)
            const int per = (nb + kThreads - 1) / kThreads;
            const int b0 = tid * per, b1 = min(nb, b0 + per);
            int64_t acc = 0;
            for (int b = b0; b < b1; ++b) acc += iabs64(vals[b]);
            int64_t incl = acc;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int64_t t = __shfl_up_sync(kFull, incl, o);
                if (lane >= o) incl += t;
            }
            if (lane == 31) warp_tot[warp] = incl;
            __syncthreads();
            int64_t woff = 0;
            for (int w = 0; w < warp; ++w) woff += warp_tot[w];
            int64_t run = woff + incl - acc;
            for (int b = b0; b < b1; ++b) {
                run += iabs64(vals[b]);
                cum[b] = run;
            }
            __syncthreads();
        }
        // index of the first bin of each 2^s-wide slice of [0, Pw): about
        // eight slices per bin, at most 1024
        int ish = 0;
        if (!learned && nb > 0) {
            const int64_t slices = nb < 128 ? 8 * nb : 1024;
            while ((Pw >> ish) >= slices) ++ish;
            const int nbk = (int)(Pw >> ish) + 1;
            for (int k = tid; k < nbk; k += kThreads) {
                const int64_t t0 = (int64_t)k << ish;
                int lo = 0, hi = nb - 1;
                while (lo < hi) {
                    const int mid = (lo + hi) >> 1;
                    if (cum[mid] > t0) hi = mid; else lo = mid + 1;
                }
                sidx[k] = (uint16_t)lo;
            }
            __syncthreads();
        }

        const int comp = it.comp;
        const int64_t m = iabs64(comp ? par.im : par.re);
        // the chunk: walkers [w_lo, w_hi) of the component, numbered in the
        // parent (real walkers first) from wb on
        const int64_t w_lo = (int64_t)it.chunk * kHeavyChunk;
        const int64_t w_hi = min(m, w_lo + kHeavyChunk);
        const int64_t wb = comp ? iabs64(par.re) : 0;
        const int64_t gw_lo = wb + w_lo, gw_hi = wb + w_hi;
        const uint2 kd = P.kd[it.seg];
        const uint32_t rank = (uint32_t)(it.parent - P.segoff[it.phase ? prv : cur][it.seg]);
        const uint32_t pre = (uint32_t)(Pw >> 20);
        // draw units: units 0 and 1 are walkers 0 and 1 (words of the rank
        // group's calls of levels 0 and 1), unit v >= 2 the parent's call
        // v - 2 (walkers 4v - 6 .. 4v - 3)
        auto unit_of = [](int64_t w) -> int64_t { return w <= 1 ? w : 2 + ((w - 2) >> 2); };
        const int64_t v_lo = unit_of(gw_lo), v_hi = unit_of(gw_hi - 1) + 1;
        for (int64_t v = v_lo + tid; v < v_hi; v += kThreads) {
            const uint4 o = v <= 1 ? group_words(rank >> 2, (uint32_t)v, it.phase, kd)
                                   : extra_words(rank, (uint32_t)(v - 2), it.phase, kd);
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                if (v <= 1 && q > 0) break;
                const int64_t w = v <= 1 ? v : 4 * v - 6 + q;
                if (w < gw_lo || w >= gw_hi) continue;
                const uint32_t W = v <= 1 ? word_of(o, (int)(rank & 3u)) : word_of(o, q);
                if (W > pre) continue;   // T >= (pre + 1) << 20 > P
                const uint32_t j = (uint32_t)(w - wb);
                const int64_t T = walker_T(W, rank, j, comp, it.phase, kd);
                if (T >= Pw) continue;
                if (learned) {
                    uint32_t V;
                    double u[2];
                    lp_draws(par.key, it.phase, comp, j, kd, &V, &u[0], &u[1]);
                    int lo = 0, hi = ns;   // first slot with cum > V
                    while (lo < hi) {
                        const int mid = (lo + hi) >> 1;
                        if (cum[mid] > (int64_t)V) hi = mid; else lo = mid + 1;
                    }
                    if (lo >= ns) continue;
                    const int64_t Qk = cum[lo] - (lo ? cum[lo - 1] : 0);
#pragma unroll
                    for (int c = 0; c < 2; ++c) {
                        const int64_t cnt = lp_count(vals[2 * lo + c], Qk, Pw, u[c]);
                        if (cnt) atomicAdd(&lh[2 * lo + c], (unsigned long long)cnt);
                    }
                    continue;
                }
                int lo = sidx[T >> ish];   // first b with cum[b] > T
                while (lo < nb - 1 && cum[lo] <= T) ++lo;
                atomicAdd(&hist[lo], 1);
            }
        }
        if (tid == 0) s_nout = 0;
        __syncthreads();
        // emit one record per nonzero (destination, channel)
        const int sg = (comp ? par.im : par.re) > 0 ? 1 : -1;
        const int sigma = it.phase ? -1 : 1;
        const int64_t init_min = P.inst[si.inst].init_min;
        const int noninit = (init_min > 0 && (iabs64(par.re) + iabs64(par.im)) < init_min) ? 1 : 0;
        if (prop)   // the remainder bins spawn nothing
            for (int b = 3 * tid + 2; b < nb; b += 3 * kThreads) hist[b] = 0;
        __syncthreads();
        auto count_of = [&](int b) -> int64_t { return learned ? (int64_t)lh[b] : (int64_t)hist[b]; };
        int my_n = 0;
        for (int b = tid; b < nb; b += kThreads) my_n += count_of(b) ? 1 : 0;
        int my_off = 0;
        if (my_n) my_off = atomicAdd(&s_nout, my_n);
        __syncthreads();
        if (tid == 0) {
            s_base = s_nout ? atomicAdd((unsigned long long*)&st->spawn_total, (unsigned long long)s_nout) : 0ull;
            if ((int64_t)s_base + s_nout > P.spawn_cap) set_error(st, DERR_SPAWN_CAPACITY);
        }
        __syncthreads();
        int k = 0;
        for (int b = tid; b < nb; b += kThreads) {
            const int64_t cnt = count_of(b);
            if (!cnt) continue;
            if (cnt > 0x7FFFFFFFll) set_error(st, DERR_POP_OVERFLOW);
            const int chan = prop ? b % 3 : (b & 1);
            const uint64_t mk = prop ? prog.stat[b / 3].mask : (learned ? prog.stat[b >> 1].mask : prog.ent[b >> 1].mask_key);
            const SRec r = make_spawn(par.key ^ mk, it.seg, comp, chan, vals[b], sg, sigma, noninit, (int32_t)cnt);
            const int64_t pos = (int64_t)s_base + my_off + k;
            if (pos < P.spawn_cap) P.spawn[pos] = r;
            ++k;
        }
        __syncthreads();
    }
}

// The plain and static-proposal kernel carries none of the learned
// proposal's state (fewer registers, more resident CTAs).
__global__ void __launch_bounds__(kThreads) k_spawn_heavy(StepParams P) { spawn_heavy<false, false>(P); }
__global__ void __launch_bounds__(kThreads) k_spawn_heavy_learned(StepParams P) { spawn_heavy<true, false>(P); }
__global__ void __launch_bounds__(kThreads) k_spawn_heavy_learned_tc(StepParams P) { spawn_heavy<true, true>(P); }

// ---------------------------------------------------------------------------
// LSD radix sort of spawn records by (segment, key).
// Digits: key bits [8p, 8p + 8) for p < key_passes, then segment bits.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t digit_of(const SRec& r, int pass, int key_passes)
{
    if (pass < key_passes) return (uint32_t)(r.key >> (8 * pass)) & 0xFFu;
    return ((r.meta >> 2) >> (8 * (pass - key_passes))) & 0xFFu;
}

__global__ void __launch_bounds__(kThreads) k_sort_hist(StepParams P)
{
    __shared__ unsigned int h[kMaxPasses * 256];
    DevState* st = P.st;
    if (cta_error(st) || !st->sort_fallback) return;
    const int64_t S = min(st->spawn_total, P.spawn_cap);
    const int np = P.key_passes + P.seg_passes;
    for (int i = threadIdx.x; i < np * 256; i += kThreads) h[i] = 0u;
    __syncthreads();
    for (int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x; i < S; i += (int64_t)gridDim.x * kThreads) {
        const SRec r = P.spawn[i];
        for (int p = 0; p < np; ++p) atomicAdd(&h[p * 256 + digit_of(r, p, P.key_passes)], 1u);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < np * 256; i += kThreads)
        if (h[i]) atomicAdd(&P.sort_hist[i], h[i]);
}

__global__ void __launch_bounds__(kThreads, 2) k_sort_scatter(StepParams P, int pass, const SRec* __restrict__ src,
                                                          SRec* __restrict__ dst)
{
    __shared__ SRec buf[kSortTile];
    __shared__ unsigned int whist[kThreads / 32][256];
    __shared__ unsigned int dbase[256];
    __shared__ unsigned int gpre[256];
    __shared__ unsigned int lstart[256];
    __shared__ unsigned int s_tile;
    DevState* st = P.st;
    if (cta_error(st) || !st->sort_fallback) return;
    const int64_t S = min(st->spawn_total, P.spawn_cap);
    const int64_t ntiles = (S + kSortTile - 1) / kSortTile;
    if (ntiles > P.sort_tiles_cap) {
        if (threadIdx.x == 0) set_error(st, DERR_TILE_CAPACITY);
        return;
    }
    const uint32_t epoch = st->seq + (uint32_t)pass;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t lt = (1u << lane) - 1u;

    // exclusive scan of the global digit histogram (once per CTA)
    {
        const unsigned int c = P.sort_hist[pass * 256 + tid];
        unsigned int incl = c;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned int t = __shfl_up_sync(kFull, incl, o);
            if (lane >= o) incl += t;
        }
        if (lane == 31) whist[0][warp] = incl;
        __syncthreads();
        unsigned int off = 0;
        for (int w = 0; w < warp; ++w) off += whist[0][w];
        dbase[tid] = off + incl - c;
        __syncthreads();
    }

    for (;;) {
        if (tid == 0) s_tile = atomicAdd(&st->tile_ctr[pass], 1u);
        __syncthreads();
        const int64_t tile = s_tile;
        if (tile >= ntiles) break;
        for (int d = tid; d < (kThreads / 32) * 256; d += kThreads) (&whist[0][0])[d] = 0u;
        __syncthreads();
        SRec rec[kSortItems];
        uint32_t dig[kSortItems];
        uint32_t rank[kSortItems];
        const int64_t t0 = tile * kSortTile;
#pragma unroll
        for (int it = 0; it < kSortItems; ++it) {
            const int64_t idx = t0 + warp * (32 * kSortItems) + it * 32 + lane;
            if (idx < S) {
                rec[it] = src[idx];
                dig[it] = digit_of(rec[it], pass, P.key_passes);
            } else {
                dig[it] = 256u;
            }
        }
        // stable warp-level ranking (warp-blocked, item-striped order = input order)
#pragma unroll
        for (int it = 0; it < kSortItems; ++it) {
            const uint32_t d = dig[it];
            const uint32_t peers = __match_any_sync(kFull, d);
            uint32_t before = 0;
            if (d < 256u) before = whist[warp][d];
            __syncwarp();
            if (d < 256u) {
                rank[it] = before + __popc(peers & lt);
                if ((peers & lt) == 0u) whist[warp][d] = before + __popc(peers);
            }
            __syncwarp();
        }
        __syncthreads();
        // per digit: warp prefixes, tile count
        unsigned int tot = 0;
        {
            const int d = tid;
            for (int w = 0; w < kThreads / 32; ++w) {
                const unsigned int c = whist[w][d];
                whist[w][d] = tot;
                tot += c;
            }
        }
        // decoupled look-back for this digit across tiles
        {
            const int d = tid;
            unsigned long long* my = P.sort_status + tile * 256 + d;
            unsigned int excl = 0;
            if (tile == 0) {
                st_vol(my, lb_word(epoch, kFlagIncl, tot));
            } else {
                st_vol(my, lb_word(epoch, kFlagAgg, tot));
                // look back 8 predecessors per probe (independent loads)
                bool done = false;
                for (int64_t hi = tile - 1; hi >= 0 && !done; hi -= 8) {
                    unsigned long long v[8];
#pragma unroll
                    for (int w = 0; w < 8; ++w) v[w] = hi - w >= 0 ? ld_vol(P.sort_status + (hi - w) * 256 + d) : 0ull;
#pragma unroll
                    for (int w = 0; w < 8; ++w) {
                        if (done || hi - w < 0) continue;
                        unsigned long long x = v[w];
                        if (!lb_ready(x, epoch)) {
                            if (!lb_wait(P.sort_status + (hi - w) * 256 + d, epoch, &x, st, 1u, hi - w, P.spin_limit)) {
                                done = true;
                                continue;
                            }
                        }
                        excl += (unsigned int)(x & kLbValMask);
                        if (lb_flag(x) == kFlagIncl) done = true;
                    }
                }
                st_vol(my, lb_word(epoch, kFlagIncl, excl + tot));
            }
            gpre[d] = excl;
        }
        // local digit starts inside the tile
        {
            unsigned int incl = tot;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const unsigned int t = __shfl_up_sync(kFull, incl, o);
                if (lane >= o) incl += t;
            }
            __shared__ unsigned int wsum[kThreads / 32];
            if (lane == 31) wsum[warp] = incl;
            __syncthreads();
            unsigned int off = 0;
            for (int w = 0; w < warp; ++w) off += wsum[w];
            lstart[tid] = off + incl - tot;
        }
        __syncthreads();
        int nvalid = 0;
#pragma unroll
        for (int it = 0; it < kSortItems; ++it) {
            if (dig[it] < 256u) {
                const uint32_t lpos = lstart[dig[it]] + whist[warp][dig[it]] + rank[it];
                buf[lpos] = rec[it];
            }
        }
        {
            const int64_t rem = S - t0;
            nvalid = (int)(rem < kSortTile ? rem : kSortTile);
        }
        __syncthreads();
        for (int j = tid; j < nvalid; j += kThreads) {
            const SRec r = buf[j];
            const uint32_t d = digit_of(r, pass, P.key_passes);
            const int64_t g = (int64_t)dbase[d] + gpre[d] + (j - (int)lstart[d]);
            if (g >= 0 && g < S) dst[g] = r;   // always true unless a look-back timed out
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// Spawn sort by buckets.  The sort key is (vector, key); its top bucket_bits
// bits (all vector bits and the top bucket_kb key bits) pick one of up to
// 2^kBucketBits buckets.  One counting pass places every spawn record in its
// bucket (order inside a bucket arbitrary).  Buckets come in sort-key order
// and each holds one vector, so sorting every bucket by key finishes the
// sort: a lane for a bucket of up to kLaneBucket records (insertion sort in
// place), a CTA for one of up to kBigBucket.  When the whole sort key fits
// the bucket digit the counting pass alone sorts.  A bucket too large for a
// CTA sends the step to the LSD radix sort instead (st->sort_fallback).
// ---------------------------------------------------------------------------
constexpr int kLaneBucket = 32;     // records a lane sorts
constexpr int kBigBucket = 4096;    // records a CTA sorts

__device__ __forceinline__ uint32_t bucket_of(const SRec& r, const StepParams& P)
{
    const uint32_t seg = r.meta >> 2;
    const int kb = P.bucket_kb;
    uint32_t d = seg << kb;
    if (kb) d |= (uint32_t)(r.key >> (2 * P.n - kb));
    return d;
}

// Bucket sizes of the step's spawn records.
__global__ void __launch_bounds__(kThreads) k_bucket_hist(StepParams P)
{
    DevState* st = P.st;
    if (read_error(st)) return;
    const int64_t S = min(st->spawn_total, P.spawn_cap);
    for (int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x; i < S; i += (int64_t)gridDim.x * kThreads)
        atomicAdd(&P.bucket[bucket_of(P.spawn[i], P)], 1u);
}

// Exclusive scan of the bucket sizes into bucket cursors: 1024 buckets per
// CTA, CTAs placed in ticket order by a decoupled look-back; decides between
// the bucket sort and the LSD fallback (a bucket above kBigBucket records).
__global__ void __launch_bounds__(1024) k_bucket_scan(StepParams P)
{
    __shared__ uint32_t wsum[32];
    __shared__ uint32_t wmax[32];
    __shared__ uint32_t s_tile;
    __shared__ unsigned long long s_excl;
    DevState* st = P.st;
    if (cta_error(st)) return;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) s_tile = atomicAdd(&st->tile_ctr[kCtrBucket], 1u);
    __syncthreads();
    const int64_t tile = s_tile;
    const int nb = 1 << P.bucket_bits;
    const int b = (int)tile * 1024 + tid;
    const uint32_t c = b < nb ? P.bucket[b] : 0u;
    uint32_t incl = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t v = __shfl_up_sync(kFull, incl, o);
        if (lane >= o) incl += v;
    }
    const uint32_t wm = __reduce_max_sync(kFull, c);
    if (lane == 31) wsum[warp] = incl;
    if (lane == 0) wmax[warp] = wm;
    __syncthreads();
    uint32_t base = 0, tot = 0, gmax = 0;
    for (int w = 0; w < 32; ++w) {
        if (w < warp) base += wsum[w];
        tot += wsum[w];
        gmax = wmax[w] > gmax ? wmax[w] : gmax;
    }
    if (warp == 0) {
        const uint32_t epoch = st->seq + 14u;
        unsigned long long* my = P.bscan_status + tile;
        unsigned long long excl = 0;
        if (tile == 0) {
            if (lane == 0) st_vol(my, lb_word(epoch, kFlagIncl, tot));
        } else {
            if (lane == 0) st_vol(my, lb_word(epoch, kFlagAgg, tot));
            excl = warp_lookback(P.bscan_status, tile, epoch, st, lane, 8u, P.spin_limit);
            if (lane == 0) st_vol(my, lb_word(epoch, kFlagIncl, excl + tot));
        }
        if (lane == 0) s_excl = excl;
    }
    __syncthreads();
    if (b < nb) {
        P.bucket[b] = (uint32_t)s_excl + base + incl - c;
    }
    if (tid == 0 && P.sort_mode == 1 && gmax > (uint32_t)kBigBucket) {
        // a bucket too large for the bucket sorts: LSD radix sort for this step
        st->sort_fallback = 1u;
        st->sort_final = (uint32_t)((P.key_passes + P.seg_passes) & 1);
    }
}

// Counting pass: spawn -> spawn_alt, each record into its bucket.  Afterwards
// bucket[b] is the end of bucket b.
__global__ void __launch_bounds__(kThreads) k_bucket_scatter(StepParams P)
{
    DevState* st = P.st;
    if (read_error(st) || st->sort_fallback) return;
    const int64_t S = min(st->spawn_total, P.spawn_cap);
    for (int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x; i < S; i += (int64_t)gridDim.x * kThreads) {
        const SRec r = P.spawn[i];
        const uint32_t pos = atomicAdd(&P.bucket[bucket_of(r, P)], 1u);
        if ((int64_t)pos < S) P.spawn_alt[pos] = r;
    }
}

// Bitonic sort (N a power of two) by (G >> 12, K): G holds the record's
// vector above its 12-bit index in the window, K its key; a window may span
// vectors.  Threads [t0, N/2) step nthr take the compare-exchanges, sync()
// orders the stages.
template <typename Sync>
__device__ __forceinline__ void bitonic_sort(uint64_t* K, uint32_t* G, int N, int t0, int nthr, Sync sync)
{
    for (int k = 2; k <= N; k <<= 1) {
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int t = t0; t < (N >> 1); t += nthr) {
                const int low = t & (j - 1);
                const int i = ((t - low) << 1) + low;   // bit j of i is clear
                const int l = i + j;
                const bool asc = (i & k) == 0;
                const uint64_t a = K[i], c = K[l];
                const uint32_t ga = G[i], gc = G[l];
                const bool gt = (ga >> 12) != (gc >> 12) ? (ga >> 12) > (gc >> 12) : a > c;
                if (gt == asc) {
                    K[i] = c;
                    K[l] = a;
                    G[i] = gc;
                    G[l] = ga;
                }
            }
            sync();
        }
    }
}

__device__ __forceinline__ int pow2_at_least(int n)
{
    int N = 2;
    while (N < n) N <<= 1;
    return N;
}

// Buckets of up to kLaneBucket records, one lane each: insertion sort by key
// in place (a bucket holds one vector; its records sit in L1 after the first
// read).  Larger buckets go to the list of k_bucket_sort_big.  After the
// counting pass bucket[b] is the end of bucket b.
__global__ void __launch_bounds__(kThreads) k_bucket_sort_small(StepParams P)
{
    DevState* st = P.st;
    if (read_error(st) || st->sort_fallback || P.sort_mode != 1) return;
    uint4* A = (uint4*)P.spawn_alt;
    const int nb = 1 << P.bucket_bits;
    for (int b = blockIdx.x * kThreads + threadIdx.x; b < nb; b += gridDim.x * kThreads) {
        const uint32_t end = P.bucket[b], start = b ? P.bucket[b - 1] : 0u;
        const int n = (int)(end - start);
        if (n <= 1) continue;
        if (n > kLaneBucket) {
            P.big_list[atomicAdd(&st->big_windows, 1u)] = (uint32_t)b;
            continue;
        }
        for (int i = 1; i < n; ++i) {
            const uint4 r = A[start + i];
            const uint64_t k = ((uint64_t)r.y << 32) | r.x;
            int j = i - 1;
            for (; j >= 0; --j) {
                const uint4 q = A[start + j];
                if ((((uint64_t)q.y << 32) | q.x) <= k) break;
                A[start + j + 1] = q;
            }
            A[start + j + 1] = r;
        }
    }
}

constexpr int kBigSortSmem = kBigBucket * (16 + 8 + 4);

// Buckets of kLaneBucket + 1 .. kBigBucket records (listed by
// k_bucket_sort_small), one CTA each.
__global__ void __launch_bounds__(kThreads) k_bucket_sort_big(StepParams P)
{
    extern __shared__ __align__(16) uint8_t bsm[];
    uint4* R = (uint4*)bsm;
    uint64_t* K = (uint64_t*)(bsm + kBigBucket * 16);
    uint32_t* G = (uint32_t*)(bsm + kBigBucket * 24);
    DevState* st = P.st;
    if (cta_error(st) || st->sort_fallback || P.sort_mode != 1) return;
    const int tid = threadIdx.x;
    const uint32_t nbig = st->big_windows;
    uint4* A = (uint4*)P.spawn_alt;
    for (uint32_t q = blockIdx.x; q < nbig; q += gridDim.x) {
        const uint32_t bk = P.big_list[q];
        const uint32_t end = P.bucket[bk], start = bk ? P.bucket[bk - 1] : 0u;
        const int n = (int)(end - start);
        if (n > kBigBucket) {   // excluded by the fallback rule
            if (tid == 0) set_error(st, DERR_TILE_CAPACITY);
            continue;
        }
        const int N = pow2_at_least(n);
        for (int j = tid; j < N; j += kThreads) {
            if (j < n) {
                const uint4 v = A[start + j];
                R[j] = v;
                K[j] = ((uint64_t)v.y << 32) | v.x;
                G[j] = ((v.z >> 2) << 12) | (uint32_t)j;
            } else {
                K[j] = ~0ull;
                G[j] = 0xFFFFF000u | (uint32_t)j;
            }
        }
        __syncthreads();
        bitonic_sort(K, G, N, tid, kThreads, [] { __syncthreads(); });
        for (int j = tid; j < n; j += kThreads) A[start + j] = R[G[j] & 0xFFFu];
        __syncthreads();
    }
}

// Offsets of each segment inside the sorted spawns (lower bounds).
// The sorted spawn records of the step (where the bucket or LSD sort left them).
__device__ __forceinline__ const SRec* sorted_spawns(const StepParams& P)
{
    return P.st->sort_final ? P.spawn_alt : P.spawn;
}

__global__ void k_spawn_segoff(StepParams P)
{
    DevState* st = P.st;
    if (read_error(st)) return;
    const SRec* __restrict__ sorted = sorted_spawns(P);
    const int64_t S = min(st->spawn_total, P.spawn_cap);
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s <= P.nseg; s += gridDim.x * blockDim.x) {
        int64_t lo = 0, hi = S;
        while (lo < hi) {
            const int64_t mid = (lo + hi) >> 1;
            if ((int)(sorted[mid].meta >> 2) < s) lo = mid + 1; else hi = mid;
        }
        P.bseg[s] = lo;
    }
}

// Merge tiles per segment (single CTA).
__global__ void k_merge_plan(StepParams P)
{
    __shared__ int64_t wsum[32];
    DevState* st = P.st;
    if (cta_error(st)) return;
    const int cur = st->cur;
    const int64_t* aoff = P.segoff[cur];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    int64_t carry = 0;
    for (int base = 0; base < P.nseg; base += blockDim.x) {
        const int s = base + tid;
        int64_t t = 0;
        if (s < P.nseg) {
            const int64_t na = aoff[s + 1] - aoff[s];
            const int64_t nb = P.bseg[s + 1] - P.bseg[s];
            t = (na + nb + kMergeTile - 1) / kMergeTile;
        }
        int64_t incl = t;
        for (int o = 1; o < 32; o <<= 1) {
            const int64_t v = __shfl_up_sync(kFull, incl, o);
            if (lane >= o) incl += v;
        }
        if (lane == 31) wsum[warp] = incl;
        __syncthreads();
        int64_t off = 0;
        for (int w = 0; w < warp; ++w) off += wsum[w];
        if (s < P.nseg) P.tile_start[s] = carry + off + incl - t;
        __syncthreads();
        int64_t blk = 0;
        for (int w = 0; w < (int)(blockDim.x / 32); ++w) blk += wsum[w];
        carry += blk;
        __syncthreads();
    }
    if (tid == 0) {
        P.tile_start[P.nseg] = carry;
        st->merge_tiles = carry;
        if (carry > st->max_tiles) st->max_tiles = carry;
        if (carry > P.merge_tiles_cap) set_error(st, DERR_TILE_CAPACITY);
    }
}

__device__ __forceinline__ int tile_seg(const int64_t* tile_start, int nseg, int64_t t)
{
    int lo = 0, hi = nseg - 1; // last s with tile_start[s] <= t
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (tile_start[mid] <= t) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// Merge-path split of one segment at diagonal d: how many of the first d
// merged items are N(t) records (ties: N(t) before spawns).
__device__ __forceinline__ int64_t merge_split(const Rec* A, const SRec* B, int64_t na, int64_t nb, int64_t d)
{
    int64_t lo = d > nb ? d - nb : 0, hi = d < na ? d : na;
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (A[mid].key <= B[d - mid - 1].key) lo = mid + 1; else hi = mid;
    }
    return lo;
}

// Metadata of every merge tile: its slices of N(t) and of the sorted spawns
// (merge-path splits at both ends) and the key just before it.
__global__ void k_merge_part(StepParams P)
{
    DevState* st = P.st;
    if (read_error(st)) return;
    const SRec* __restrict__ sorted = sorted_spawns(P);
    const int cur = st->cur;
    const int64_t T = st->merge_tiles;
    const Rec* A = P.pop[cur];
    const int64_t* aoff = P.segoff[cur];
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < T; t += (int64_t)gridDim.x * blockDim.x) {
        const int s = tile_seg(P.tile_start, P.nseg, t);
        const int64_t a0 = aoff[s], na = aoff[s + 1] - a0;
        const int64_t b0 = P.bseg[s], nb = P.bseg[s + 1] - b0;
        const int64_t d = (t - P.tile_start[s]) * kMergeTile;
        const int64_t d1 = min(d + (int64_t)kMergeTile, na + nb);
        const int64_t ia0 = merge_split(A + a0, sorted + b0, na, nb, d), ib0 = d - ia0;
        const int64_t ia1 = merge_split(A + a0, sorted + b0, na, nb, d1), ib1 = d1 - ia1;
        uint64_t pk = 0;
        if (ia0 > 0) pk = A[a0 + ia0 - 1].key;
        if (ib0 > 0) {
            const uint64_t kb = sorted[b0 + ib0 - 1].key;
            pk = pk > kb ? pk : kb;
        }
        MTileG g;
        g.a_glob = a0 + ia0;
        g.b_glob = b0 + ib0;
        g.b_seg_end = b0 + nb;
        g.prev_key = pk;
        g.na = (int32_t)(ia1 - ia0);
        g.nb = (int32_t)(ib1 - ib0);
        g.seg = s;
        g.has_prev = (ia0 > 0 || ib0 > 0) ? 1 : 0;
        P.mtiles[t] = g;
    }
}

// ---------------------------------------------------------------------------
// Annihilation [End Matter, annihilation step].  A run is all items (at most
// one N(t) record and any number of spawn records) with one key.  Value =
// N(t) + initiator spawns + (occupied ? non-initiator spawns : 0); zero runs
// are dropped.  A producer warp stages the tiles of the merged sequence in
// shared memory by bulk copies (two stages); each of the 256 merging threads
// merges kMergeItems items and emits the runs whose first item it holds,
// reading past its items (and past the tile, where only spawn records can
// follow, since N(t) sorts first on equal keys) to finish its last run.  The
// tile's runs are compacted in shared memory; a publisher warp places them by
// a decoupled look-back over the tiles and writes them out with one bulk
// store, while the merging warps go on with the next tile.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint64_t it_key(const uint4* buf, int i)
{
    return ((const uint64_t*)&buf[i])[0];
}

// Walk the thread's items of a tile; the runs it owns go to raw[0 ..),
// their statistics to ntot / dre / dim.  Returns the number of runs.
__device__ __forceinline__ int merge_walk(const uint4* buf, const MTileG& m, const SRec* __restrict__ sorted,
                                          uint4* raw, DevState* st, uint32_t n, uint32_t ymask, long long* ntot,
                                          long long* dre, long long* dim, long long* zrow)
{
    const int na = m.na, nb = m.nb, nt = na + nb;
    const int d0 = (int)threadIdx.x * kMergeItems;
    if (d0 >= nt) return 0;
    int lo = d0 > nb ? d0 - nb : 0, hi = d0 < na ? d0 : na;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (it_key(buf, mid) <= it_key(buf, na + d0 - mid - 1)) lo = mid + 1; else hi = mid;
    }
    int ia = lo, ib = d0 - lo;
    bool has_prev;
    uint64_t prev;
    if (d0 == 0) {
        has_prev = m.has_prev != 0;
        prev = m.prev_key;
    } else {
        has_prev = true;
        const uint64_t ka = ia > 0 ? it_key(buf, ia - 1) : 0ull;
        const uint64_t kb = ib > 0 ? it_key(buf, na + ib - 1) : 0ull;
        prev = ka > kb ? ka : kb;
    }
    const int cnt = min(kMergeItems, nt - d0);
    int nout = 0;
    bool open = false, occupied = false;
    uint64_t rkey = 0;
    long long sre = 0, sim = 0, nre = 0, nim = 0;
    auto close_run = [&]() {
        long long vr = sre, vi = sim;
        if (occupied) { vr += nre; vi += nim; }
        if (vr == 0 && vi == 0) return;
        if (vr > 2147483647ll || vr < -2147483647ll || vi > 2147483647ll || vi < -2147483647ll) {
            set_error(st, DERR_POP_OVERFLOW);
            return;
        }
        *ntot += (vr < 0 ? -vr : vr) + (vi < 0 ? -vi : vi);
        if ((uint32_t)(rkey >> n) == (uint32_t)(rkey & ymask)) {
            *dre += vr;
            *dim += vi;
            // <Z_q> on the diagonal: Re N_xx of the states with bit q of x set
            // (zrow: the tile's sums in shared memory)
            for (uint32_t xb = (uint32_t)(rkey >> n); xb; xb &= xb - 1u)
                atomicAdd((unsigned long long*)&zrow[__ffs(xb) - 1], (unsigned long long)vr);
        }
        raw[nout] = make_uint4((uint32_t)rkey, (uint32_t)(rkey >> 32), (uint32_t)(int32_t)vr, (uint32_t)(int32_t)vi);
        ++nout;
    };
    auto add_item = [&](int idx, bool isA) {
        const uint4 w = buf[idx];
        if (isA) {
            occupied = true;
            sre += (int32_t)w.z;
            sim += (int32_t)w.w;
        } else {
            const uint32_t meta = w.z;
            const long long v = (int32_t)w.w;
            if (meta & 1u) { if (meta & 2u) nim += v; else nre += v; }
            else { if (meta & 2u) sim += v; else sre += v; }
        }
    };
    bool leading = true;
    for (int k = 0; k < cnt; ++k) {
        bool takeA;
        if (ia >= na) takeA = false;
        else if (ib >= nb) takeA = true;
        else takeA = it_key(buf, ia) <= it_key(buf, na + ib);
        const int idx = takeA ? ia++ : na + ib++;
        const uint64_t key = it_key(buf, idx);
        if (leading) {
            if (has_prev && key == prev) continue; // run owned by an earlier thread or tile
            leading = false;
        }
        if (open && key == rkey) {
            add_item(idx, takeA);
            continue;
        }
        if (open) close_run();
        open = true;
        occupied = false;
        rkey = key;
        sre = sim = nre = nim = 0;
        add_item(idx, takeA);
    }
    if (open) {
        // finish the last run: later items of this tile, then spawns past the
        // tile.  Every item before the run's next one has a key <= rkey, and
        // N(t) sorts first on equal keys, so an N(t) record of key rkey would
        // come first, then the tile's spawns of key rkey, a stretch from ib
        // (they ascend from rkey): its end by a galloping search, then a sum
        // over the stretch whose loads do not wait on one another (long runs
        // come from concentrated spawns).
        if (ia < na && it_key(buf, ia) == rkey) {
            add_item(ia, true);
            ++ia;
        }
        {
            int lo = ib, hi = ib, step = 1;   // the tile's spawns [ib, lo) carry rkey
            while (hi < nb && it_key(buf, na + hi) == rkey) {
                lo = hi + 1;
                hi = min(nb, ib + 2 * step - 1);
                step *= 2;
            }
            while (lo < hi) {
                const int mid = (lo + hi) >> 1;
                if (it_key(buf, na + mid) == rkey) lo = mid + 1; else hi = mid;
            }
            for (int j = ib; j < lo; ++j) add_item(na + j, false);
            ib = lo;
        }
        if (ia >= na && ib >= nb) {
            // the run's spawns past the tile (their keys ascend from rkey): the
            // run's end by a galloping search, then a sum over that range whose
            // loads do not wait on one another (runs of thousands of records
            // come from heavy parents' chunks)
            const int64_t j0 = m.b_glob + nb, j1 = m.b_seg_end;
            int64_t lo = j0, hi = j0, step = 1;   // every key in [j0, lo) is rkey
            while (hi < j1 && sorted[hi].key == rkey) {
                lo = hi + 1;
                hi = min(j1, j0 + 2 * step - 1);
                step *= 2;
            }
            while (lo < hi) {   // the first index in [lo, hi) whose key is above rkey
                const int64_t mid = (lo + hi) >> 1;
                if (sorted[mid].key == rkey) lo = mid + 1; else hi = mid;
            }
            for (int64_t jb = j0; jb < lo; ++jb) {
                const SRec r = sorted[jb];
                const long long v = r.val;
                if (r.meta & 1u) { if (r.meta & 2u) nim += v; else nre += v; }
                else { if (r.meta & 2u) sim += v; else sre += v; }
            }
        }
        close_run();
    }
    return nout;
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}

// Barrier of the 256 merging threads only (the producer warp runs apart).
__device__ __forceinline__ void merge_bar()
{
    asm volatile("bar.sync 1, %0;" ::"n"(kThreads) : "memory");
}

// 1-D bulk copy shared -> global (bulk async-group); both addresses 16-byte
// aligned, bytes a multiple of 16.
__device__ __forceinline__ void bulk_store(void* dst, const void* src, uint32_t bytes)
{
    asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(dst), "r"(smem_addr(src)),
                 "r"(bytes)
                 : "memory");
    asm volatile("cp.async.bulk.commit_group;" ::: "memory");
}

// Shared memory: kMergeStages input stages (each also holds its tile's
// compacted output until the bulk store has read it) and one buffer of raw
// runs (kMergeTile 16-byte items each).
constexpr int kMergeStages = 4;
constexpr int kMergeSmem = (kMergeStages + 1) * kMergeTile * 16;

// Per-tile hand-over from the merging warps to the publisher warp.
struct MSlot {
    int64_t t;
    long long ntot, dre, dim;
    int32_t count, seg;
};

// Warp roles: 0..7 merge, 8 produces (tickets, bulk loads), 9 publishes
// (look-back, statistics, bulk store of the compacted output).
__global__ void __launch_bounds__(kMergeThreads, 2) k_merge(StepParams P)
{
    extern __shared__ __align__(128) uint4 msm[];
    uint4* inbuf = msm;                                // [kMergeStages][kMergeTile]
    uint4* raw = msm + kMergeStages * kMergeTile;      // [kMergeTile]
    __shared__ __align__(8) uint64_t full[kMergeStages], empty[kMergeStages], ready[kMergeStages];
    __shared__ MTileG meta[kMergeStages];
    __shared__ int64_t meta_t[kMergeStages];
    __shared__ MSlot slot[kMergeStages];
    __shared__ int s_wcount[2][kThreads / 32];
    __shared__ long long s_red[2][3][kThreads / 32];
    __shared__ int s_abort;
    __shared__ long long s_z[32];   // the tile's <Z_q> sums, added to its vector's once per tile
    DevState* st = P.st;
    if (cta_error(st)) return;
    const int cur = st->cur, nxt = (cur + 1) % 3;
    const int64_t T = st->merge_tiles;
    const SRec* __restrict__ sorted = sorted_spawns(P);
    const Rec* A = P.pop[cur];
    Rec* out = P.pop[nxt];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    constexpr int kMergeWarps = kThreads / 32;
    if (tid == 0) {
        for (int s = 0; s < kMergeStages; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
            mbar_init(&ready[s], kMergeWarps);
        }
        mbar_fence_init();
        s_abort = 0;
    }
    __syncthreads();

    if (warp == kMergeWarps) {
        // producer: take tiles in order (one ticket each), stage them
        if (lane != 0) return;
        int issued[kMergeStages] = {};
        int end_stage = -1;
        for (int k = 0;; ++k) {
            const int s = k % kMergeStages;
            if (k >= kMergeStages && !mbar_wait(&empty[s], (uint32_t)((k / kMergeStages - 1) & 1), st, 3u, k))
                break;
            const int64_t t = (int64_t)atomicAdd(&st->tile_ctr[kCtrMerge], 1u);
            meta_t[s] = t;
            if (t >= T) {
                mbar_arrive(&full[s]);   // end marker
                end_stage = s;
                break;
            }
            const MTileG m = P.mtiles[t];
            meta[s] = m;
            const uint32_t abytes = (uint32_t)m.na * 16u, bbytes = (uint32_t)m.nb * 16u;
            fence_proxy_async();
            mbar_arrive_expect(&full[s], abytes + bbytes);
            if (abytes) bulk_load(inbuf + s * kMergeTile, A + m.a_glob, abytes, &full[s]);
            if (bbytes) bulk_load(inbuf + s * kMergeTile + m.na, sorted + m.b_glob, bbytes, &full[s]);
            ++issued[s];
        }
        // No copy may still be writing shared memory when the CTA exits.  The
        // end marker goes to a stage only after its last copy was consumed
        // (and its phase parity no longer names that copy); on the other
        // stage the last copy's phase is the current or the previous one.
        for (int s = 0; s < kMergeStages; ++s)
            if (issued[s] && s != end_stage) mbar_wait(&full[s], (uint32_t)((issued[s] - 1) & 1), st, 4u, s);
        return;
    }

    const uint32_t epoch = st->seq + 15u;
    if (warp == kMergeWarps + 1) {
        // publisher: place each tile after its predecessors (the merging
        // warps published its aggregate), store it.  A stage is released once
        // its bulk store has read it: right away when the tile stores
        // nothing, else after the next store is issued.
        int pending = -1;
        for (int k = 0;; ++k) {
            const int s = k % kMergeStages;
            if (!mbar_wait(&ready[s], (uint32_t)((k / kMergeStages) & 1), st, 6u, k)) break;
            const MSlot sl = slot[s];
            if (sl.t >= T) break;
            unsigned long long excl = 0;
            if (sl.t > 0) {
                excl = warp_lookback(P.merge_status, sl.t, epoch, st, lane, 2u, P.spin_limit);
                if (lane == 0) st_vol(P.merge_status + sl.t, lb_word(epoch, kFlagIncl, excl + (unsigned long long)sl.count));
            }
            if (lane == 0) {
                if (sl.t == T - 1) {
                    st->next_total = (int64_t)(excl + sl.count);
                    if ((int64_t)(excl + sl.count) > st->max_next) st->max_next = (int64_t)(excl + sl.count);
                }
                bool stored = false;
                if (sl.count) {
                    atomicAdd(&P.segacc[sl.seg].count, (unsigned long long)sl.count);
                    atomicAdd((unsigned long long*)&P.segacc[sl.seg].ntot, (unsigned long long)sl.ntot);
                    atomicAdd((unsigned long long*)&P.segacc[sl.seg].dre, (unsigned long long)sl.dre);
                    atomicAdd((unsigned long long*)&P.segacc[sl.seg].dim, (unsigned long long)sl.dim);
                    const int64_t base = (int64_t)excl;
                    int64_t cnt = sl.count;
                    if (base + cnt > P.pop_cap) {
                        set_error(st, DERR_POP_CAPACITY);
                        cnt = base < P.pop_cap ? P.pop_cap - base : 0;
                    }
                    if (cnt > 0) {
                        bulk_store(out + base, inbuf + s * kMergeTile, (uint32_t)cnt * 16u);
                        stored = true;
                    }
                }
                if (stored) {
                    asm volatile("cp.async.bulk.wait_group.read 1;" ::: "memory");
                    if (pending >= 0) mbar_arrive(&empty[pending]);
                    pending = s;
                } else {
                    asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
                    if (pending >= 0) mbar_arrive(&empty[pending]);
                    pending = -1;
                    mbar_arrive(&empty[s]);
                }
            }
            __syncwarp();
        }
        if (lane == 0) asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
        return;
    }

    // merging threads
    if (tid < 32) s_z[tid] = 0ll;
    merge_bar();
    for (int k = 0;; ++k) {
        const int s = k % kMergeStages, h = k & 1;
        const bool ok = mbar_wait(&full[s], (uint32_t)((k / kMergeStages) & 1), st, 5u, k);
        if (!ok) s_abort = 1;
        const int64_t t = ok ? meta_t[s] : T;
        long long my_ntot = 0, my_dre = 0, my_dim = 0;
        int nout = 0;
        int seg = 0;
        if (t < T) {
            const MTileG m = meta[s];
            seg = m.seg;
            const uint32_t n = (uint32_t)P.seginfo[seg].n;   // the tile's vector's qubit count
            const uint32_t ymask = n == 32 ? 0xFFFFFFFFu : ((1u << n) - 1u);
            nout = merge_walk(inbuf + s * kMergeTile, m, sorted, raw + tid * kMergeItems, st, n, ymask, &my_ntot,
                              &my_dre, &my_dim, s_z);
        }
        // block scan of run counts, block sums of the statistics
        int incl = nout;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int v = __shfl_up_sync(kFull, incl, o);
            if (lane >= o) incl += v;
        }
        if (lane == 31) s_wcount[h][warp] = incl;
        long long r0 = my_ntot, r1 = my_dre, r2 = my_dim;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            r0 += __shfl_down_sync(kFull, r0, o);
            r1 += __shfl_down_sync(kFull, r1, o);
            r2 += __shfl_down_sync(kFull, r2, o);
        }
        if (lane == 0) {
            s_red[h][0][warp] = r0;
            s_red[h][1][warp] = r1;
            s_red[h][2][warp] = r2;
        }
        merge_bar();   // walks of the tile done, counts known
        if (s_abort || t >= T) {
            // tell the publisher to stop
            if (tid == 0) slot[s].t = T;
            __syncwarp();
            if (lane == 0) mbar_arrive(&ready[s]);
            break;
        }
        if (tid < 32) {   // the tile's <Z_q> sums to its vector's (the walks are done)
            const long long z = s_z[tid];
            if (z) {
                atomicAdd((unsigned long long*)&P.zacc[32 * (int64_t)seg + tid], (unsigned long long)z);
                s_z[tid] = 0ll;
            }
        }
        int woff = 0, tile_count = 0;
#pragma unroll
        for (int w = 0; w < kMergeWarps; ++w) {
            if (w < warp) woff += s_wcount[h][w];
            tile_count += s_wcount[h][w];
        }
        // compact the runs over the consumed input stage
        uint4* ob = inbuf + s * kMergeTile;
        const int pos = woff + incl - nout;
        for (int r = 0; r < nout; ++r) ob[pos + r] = raw[tid * kMergeItems + r];
        fence_proxy_async();   // generic writes of ob before the bulk store reads them
        merge_bar();           // raw runs read before the next walk rewrites them
        if (tid == 0) {
            // the tile's aggregate (inclusive prefix for the first tile), at once
            st_vol(P.merge_status + t, lb_word(epoch, t == 0 ? kFlagIncl : kFlagAgg, (unsigned long long)tile_count));
            MSlot sl;
            sl.t = t;
            sl.count = tile_count;
            sl.seg = seg;
            sl.ntot = sl.dre = sl.dim = 0;
            for (int w = 0; w < kMergeWarps; ++w) {
                sl.ntot += s_red[h][0][w];
                sl.dre += s_red[h][1][w];
                sl.dim += s_red[h][2][w];
            }
            slot[s] = sl;
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&ready[s]);
    }
}

// Segment offsets of N(t + dt), history, rotation (single CTA).
__global__ void k_finalize(StepParams P)
{
    __shared__ long long wsum[32];
    DevState* st = P.st;
    if (cta_error(st)) return;
    const int cur = st->cur, nxt = (cur + 1) % 3;
    int64_t* off = P.segoff[nxt];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int ci = st->call_index;
    long long carry = 0;
    for (int base = 0; base < P.nseg; base += blockDim.x) {
        const int s = base + tid;
        long long c = 0;
        if (s < P.nseg) {
            c = (long long)P.segacc[s].count;
            if (ci < P.history_cap) {
                SegStats h = P.segacc[s];
                P.history[(int64_t)ci * P.nseg + s] = h;
                // N^diag <Z_q> = sum of Re N_xx (-1)^(x_q) = Re N^diag - 2 (the part with bit q set)
                const int nq = P.seginfo[s].n;
                long long* zh = P.zhist + ((int64_t)ci * P.nseg + s) * P.n;
                for (int q = 0; q < P.n; ++q) zh[q] = q < nq ? h.dre - 2 * P.zacc[32 * (int64_t)s + q] : 0ll;
            }
        }
        long long incl = c;
        for (int o = 1; o < 32; o <<= 1) {
            const long long v = __shfl_up_sync(kFull, incl, o);
            if (lane >= o) incl += v;
        }
        if (lane == 31) wsum[warp] = incl;
        __syncthreads();
        long long wo = 0;
        for (int w = 0; w < warp; ++w) wo += wsum[w];
        if (s < P.nseg) off[s] = carry + wo + incl - c;
        __syncthreads();
        long long blk = 0;
        for (int w = 0; w < (int)(blockDim.x / 32); ++w) blk += wsum[w];
        carry += blk;
        __syncthreads();
    }
    if (tid == 0) {
        long long walkers = 0;
        for (int s = 0; s < P.nseg; ++s) walkers += P.segacc[s].ntot;
        const StepInfo inf = P.info[ci];
        st->acc_steps += 1;
        st->acc_walkers += walkers;
        st->acc_kcur += st->count[cur];
        st->acc_kprev += inf.ab2 ? st->count[(cur + 2) % 3] : 0;
        st->acc_spawn += st->spawn_total;
        st->acc_knext += carry;
        st->acc_heavy += st->heavy_total;
        st->acc_cand += st->cand_total;
        if (st->sort_fallback) st->acc_sort_lsd += 1; else st->acc_sort_bucket += 1;
        off[P.nseg] = carry;
        if (st->spawn_total > st->max_spawn) st->max_spawn = st->spawn_total;
        if (st->cand_total > st->max_cand) st->max_cand = st->cand_total;
        if (st->heavy_total > st->max_heavy) st->max_heavy = st->heavy_total;
        st->count[nxt] = carry;
        st->cur = nxt;
        st->step += 1;
        st->call_index += 1;
    }
}

// ---------------------------------------------------------------------------
// Initial populations: N(0) = N^diag rho(0), stochastic rounding per
// component with the kind-1 stream of each segment.
// ---------------------------------------------------------------------------
// Key of element (x, y) of rho(0) in a vector of n qubits.
__device__ __forceinline__ uint64_t init_key(const uint64_t* x, const uint64_t* y, int64_t e, int n)
{
    return (x[e] << n) | y[e];
}

__global__ void k_init_values(StepParams P, const uint64_t* __restrict__ xs, const uint64_t* __restrict__ ys,
                              const double* __restrict__ re, const double* __restrict__ im, int64_t nnz,
                              int64_t* __restrict__ vals)
{
    const int64_t total = nnz * P.nseg;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const int s = (int)(i / nnz);
        const int64_t e = i - (int64_t)s * nnz;
        const SegInfo si = P.seginfo[s];
        const InstInfo in = P.inst[si.inst];
        const int64_t n_diag = in.n_diag;
        const uint4 kk = philox10(make_uint4(0u, 0u, (uint32_t)si.vec, kTagInit),
                                  make_uint2((uint32_t)in.seed, (uint32_t)(in.seed >> 32)));
        const uint2 kd = make_uint2(kk.x, kk.y);
        const uint64_t key = init_key(xs, ys, e, si.n);
        for (int comp = 0; comp < 2; ++comp) {
            const double v = __dmul_rn((double)n_diag, comp ? im[e] : re[e]);
            const double fl = floor(v);
            const double fr = __dsub_rn(v, fl);
            const uint4 w = philox10(make_uint4((uint32_t)key, (uint32_t)(key >> 32),
                                                ((uint32_t)comp << 1) | (kKindInit << 2), 0u), kd);
            const uint64_t r = ((uint64_t)w.y << 32) | w.x;
            const double u = __dmul_rn((double)(r >> 11), 1.0 / 9007199254740992.0);
            int64_t val = (int64_t)fl + (u < fr ? 1 : 0);
            if (val > 2147483647ll || val < -2147483647ll) {
                set_error(P.st, DERR_POP_OVERFLOW);
                val = 0;
            }
            vals[2 * i + comp] = val;
        }
    }
}

// Compact nonzero values per segment into slot 'cur' (single CTA, in order).
__global__ void k_init_compact(StepParams P, const uint64_t* __restrict__ xs, const uint64_t* __restrict__ ys,
                               int64_t nnz, const int64_t* __restrict__ vals)
{
    __shared__ int s_cnt[kThreads];
    DevState* st = P.st;
    const int slot = st->cur;
    Rec* dst = P.pop[slot];
    int64_t* off = P.segoff[slot];
    int64_t pos = 0;
    const int tid = threadIdx.x;
    for (int s = 0; s < P.nseg; ++s) {
        if (tid == 0) off[s] = pos;
        for (int64_t base = 0; base < nnz; base += kThreads) {
            const int64_t e = base + tid;
            const int64_t i = (int64_t)s * nnz + e;
            const bool keep = e < nnz && (vals[2 * i] != 0 || vals[2 * i + 1] != 0);
            s_cnt[tid] = keep ? 1 : 0;
            __syncthreads();
            for (int o = 1; o < kThreads; o <<= 1) {
                const int v = tid >= o ? s_cnt[tid - o] : 0;
                __syncthreads();
                s_cnt[tid] += v;
                __syncthreads();
            }
            const int excl = s_cnt[tid] - (keep ? 1 : 0);
            const int blk = s_cnt[kThreads - 1];
            if (keep && pos + excl < P.pop_cap)
                dst[pos + excl] = Rec{init_key(xs, ys, e, P.seginfo[s].n), (int32_t)vals[2 * i], (int32_t)vals[2 * i + 1]};
            pos += blk;
            __syncthreads();
        }
    }
    if (tid == 0) {
        off[P.nseg] = pos;
        st->count[slot] = pos;
        if (pos > P.pop_cap) set_error(st, DERR_POP_CAPACITY);
    }
}

// Per-segment K, N_tot, N^diag of one population slot.  Each block takes a
// contiguous range; a thread accumulates while its segment stays the same and
// flushes with atomics when it changes (records are sorted by segment).
__global__ void k_obs(StepParams P, int which, SegStats* __restrict__ out)
{
    const DevState* st = P.st;
    const int slot = which == 0 ? st->cur : (st->cur + 2) % 3;
    const Rec* pop = P.pop[slot];
    const int64_t* off = P.segoff[slot];
    const int64_t K = off[P.nseg];
    int n = 32;
    uint32_t ymask = 0xFFFFFFFFu;
    const int64_t per = (K + gridDim.x - 1) / gridDim.x;
    const int64_t b0 = (int64_t)blockIdx.x * per, b1 = min(K, b0 + per);
    int cs = -1;
    int64_t cs_end = 0;
    unsigned long long c = 0;
    long long ntot = 0, dre = 0, dim = 0;
    auto flush = [&]() {
        if (cs < 0 || c == 0) return;
        atomicAdd(&out[cs].count, c);
        atomicAdd((unsigned long long*)&out[cs].ntot, (unsigned long long)ntot);
        atomicAdd((unsigned long long*)&out[cs].dre, (unsigned long long)dre);
        atomicAdd((unsigned long long*)&out[cs].dim, (unsigned long long)dim);
    };
    for (int64_t i = b0 + threadIdx.x; i < b1; i += blockDim.x) {
        if (cs < 0 || i >= cs_end) {
            flush();
            cs = seg_of(off, P.nseg, i);
            cs_end = off[cs + 1];
            n = P.seginfo[cs].n;
            ymask = n == 32 ? 0xFFFFFFFFu : ((1u << n) - 1u);
            c = 0;
            ntot = dre = dim = 0;
        }
        const Rec r = pop[i];
        ++c;
        ntot += (r.re < 0 ? -(long long)r.re : r.re) + (r.im < 0 ? -(long long)r.im : r.im);
        if ((uint32_t)(r.key >> n) == (uint32_t)(r.key & ymask)) {
            dre += r.re;
            dim += r.im;
        }
    }
    flush();
}

// Values of query keys in one segment of N(t) (0 when absent).
__global__ void k_lookup(StepParams P, int seg, const uint64_t* __restrict__ q, int nq, int64_t* __restrict__ out)
{
    const DevState* st = P.st;
    const int slot = st->cur;
    const Rec* pop = P.pop[slot];
    const int64_t lo0 = P.segoff[slot][seg], hi0 = P.segoff[slot][seg + 1];
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nq; i += gridDim.x * blockDim.x) {
        int64_t lo = lo0, hi = hi0;
        const uint64_t key = q[i];
        while (lo < hi) {
            const int64_t mid = (lo + hi) >> 1;
            if (pop[mid].key < key) lo = mid + 1; else hi = mid;
        }
        int64_t re = 0, im = 0;
        if (lo < hi0 && pop[lo].key == key) { re = pop[lo].re; im = pop[lo].im; }
        out[2 * i] = re;
        out[2 * i + 1] = im;
    }
}

// Overlap of every vector of N(t) with a target |psi> given on len basis
// states idx[a] (psi as (re, im) pairs): sum over a, b of conj(psi_a) N_ab
// psi_b [fidelity, Markovian circuit dynamics], one CTA per vector.  The
// values N_ab are looked up exactly; the sum runs in one thread in the fixed
// order (a, then b) with every product and sum rounded as written.
__global__ void k_overlap_all(StepParams P, const uint64_t* __restrict__ idx, const double* __restrict__ psi, int len,
                              double* __restrict__ out)
{
    __shared__ long long v[2 * kMaxOverlapLen * kMaxOverlapLen];
    const DevState* st = P.st;
    const int slot = st->cur;
    const int seg = blockIdx.x;
    const Rec* pop = P.pop[slot];
    const int64_t lo0 = P.segoff[slot][seg], hi0 = P.segoff[slot][seg + 1];
    const int n = P.seginfo[seg].n;
    for (int e = threadIdx.x; e < len * len; e += blockDim.x) {
        const uint64_t key = (idx[e / len] << n) | idx[e % len];
        int64_t lo = lo0, hi = hi0;
        while (lo < hi) {
            const int64_t mid = (lo + hi) >> 1;
            if (pop[mid].key < key) lo = mid + 1; else hi = mid;
        }
        long long re = 0, im = 0;
        if (lo < hi0 && pop[lo].key == key) {
            re = pop[lo].re;
            im = pop[lo].im;
        }
        v[2 * e] = re;
        v[2 * e + 1] = im;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double sr = 0.0, si = 0.0;
        for (int a = 0; a < len; ++a) {
            for (int b = 0; b < len; ++b) {
                const double nr = (double)v[2 * (a * len + b)], ni = (double)v[2 * (a * len + b) + 1];
                const double car = psi[2 * a], cai = -psi[2 * a + 1];
                const double pr = __dsub_rn(__dmul_rn(car, nr), __dmul_rn(cai, ni));
                const double pi = __dadd_rn(__dmul_rn(car, ni), __dmul_rn(cai, nr));
                sr = __dadd_rn(sr, __dsub_rn(__dmul_rn(pr, psi[2 * b]), __dmul_rn(pi, psi[2 * b + 1])));
                si = __dadd_rn(si, __dadd_rn(__dmul_rn(pr, psi[2 * b + 1]), __dmul_rn(pi, psi[2 * b])));
            }
        }
        out[2 * seg] = sr;
        out[2 * seg + 1] = si;
    }
}

// Add a non-negative 128-bit value to a (low, high) pair of 64-bit words.
__device__ __forceinline__ void add_u128(unsigned long long* w, unsigned __int128 v)
{
    const unsigned long long lo = (unsigned long long)v;
    unsigned long long hi = (unsigned long long)(v >> 64);
    if (lo) {
        const unsigned long long old = atomicAdd(&w[0], lo);
        if (old + lo < old) ++hi;   // carry out of the low word
    }
    if (hi) atomicAdd(&w[1], hi);
}

// ||N - N^dagger||_F^2 of every vector of N(t) [End Matter on Hermiticity
// preservation], exactly: each record contributes |N_xy - conj(N_yx)|^2 (the
// transposed record found by binary search in its vector; the diagonal is its
// own transpose) and, when the transposed state is unoccupied, also the
// transposed entry's |N_xy|^2.  Each CTA takes a contiguous range of records;
// a thread's sums go out once per vector it leaves.
__global__ void k_antiherm(StepParams P, unsigned long long* __restrict__ out)
{
    const DevState* st = P.st;
    const int slot = st->cur;
    const Rec* pop = P.pop[slot];
    const int64_t* off = P.segoff[slot];
    const int64_t K = off[P.nseg];
    const int64_t per = (K + gridDim.x - 1) / gridDim.x;
    const int64_t b0 = (int64_t)blockIdx.x * per, b1 = min(K, b0 + per);
    int cs = -1, n = 32;
    int64_t cs_lo = 0, cs_end = 0;
    unsigned __int128 acc = 0;
    for (int64_t i = b0 + threadIdx.x; i < b1; i += blockDim.x) {
        if (cs < 0 || i >= cs_end) {
            if (cs >= 0 && acc) add_u128(out + 2 * cs, acc);
            acc = 0;
            cs = seg_of(off, P.nseg, i);
            cs_lo = off[cs];
            cs_end = off[cs + 1];
            n = P.seginfo[cs].n;
        }
        const Rec r = pop[i];
        const uint64_t ymask = n == 32 ? 0xFFFFFFFFull : ((1ull << n) - 1ull);
        const uint64_t x = r.key >> n, y = r.key & ymask;
        const uint64_t tk = (y << n) | x;
        long long tre = 0, tim = 0;
        if (tk == r.key) {
            tre = r.re;
            tim = r.im;
        } else {
            int64_t lo = cs_lo, hi = cs_end;
            while (lo < hi) {
                const int64_t mid = (lo + hi) >> 1;
                if (pop[mid].key < tk) lo = mid + 1; else hi = mid;
            }
            if (lo < cs_end && pop[lo].key == tk) {
                tre = pop[lo].re;
                tim = pop[lo].im;
            }
        }
        const long long dre = (long long)r.re - tre, dim = (long long)r.im + tim;
        acc += (unsigned __int128)((__int128)dre * dre) + (unsigned __int128)((__int128)dim * dim);
        if (tre == 0 && tim == 0)
            acc += (unsigned __int128)((__int128)r.re * r.re) + (unsigned __int128)((__int128)r.im * r.im);
    }
    if (cs >= 0 && acc) add_u128(out + 2 * cs, acc);
}

// Value of N(t) at key in vector seg (0 when unoccupied), by binary search.
__device__ __forceinline__ void value_in(const Rec* pop, const int64_t* off, int seg, uint64_t key, long long* re,
                                         long long* im)
{
    int64_t lo = off[seg], hi = off[seg + 1];
    const int64_t end = hi;
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (pop[mid].key < key) lo = mid + 1; else hi = mid;
    }
    *re = 0;
    *im = 0;
    if (lo < end && pop[lo].key == key) {
        *re = pop[lo].re;
        *im = pop[lo].im;
    }
}

// ||S - S^dagger||_F^2 of the sum S of the listed vectors of N(t), exactly
// (the replica aggregate's anti-Hermiticity).  Grid (x: records, y: listed
// vector a).  A record (x, y) of vector segs[a] accounts for the entry (x, y)
// when no earlier listed vector holds (x, y), and then also for the entry
// (y, x) when no listed vector holds (y, x).
__global__ void k_antiherm_sum(StepParams P, const int32_t* __restrict__ segs, int count,
                               unsigned long long* __restrict__ out)
{
    const DevState* st = P.st;
    const int slot = st->cur;
    const Rec* pop = P.pop[slot];
    const int64_t* off = P.segoff[slot];
    const int a = blockIdx.y;
    const int sa = segs[a];
    const int n = P.seginfo[sa].n;
    const uint64_t ymask = n == 32 ? 0xFFFFFFFFull : ((1ull << n) - 1ull);
    unsigned __int128 acc = 0;
    for (int64_t i = off[sa] + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < off[sa + 1];
         i += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t key = pop[i].key;
        const uint64_t tkey = ((key & ymask) << n) | (key >> n);
        bool first = true;
        for (int b = 0; b < a && first; ++b) {
            long long re, im;
            value_in(pop, off, segs[b], key, &re, &im);
            if (re != 0 || im != 0) first = false;
        }
        if (!first) continue;
        long long sre = 0, sim = 0, tre = 0, tim = 0;
        bool t_held = false;
        for (int b = 0; b < count; ++b) {
            long long re, im;
            value_in(pop, off, segs[b], key, &re, &im);
            sre += re;
            sim += im;
            value_in(pop, off, segs[b], tkey, &re, &im);
            tre += re;
            tim += im;
            t_held |= re != 0 || im != 0;
        }
        const long long dre = sre - tre, dim = sim + tim;
        acc += (unsigned __int128)((__int128)dre * dre) + (unsigned __int128)((__int128)dim * dim);
        if (tkey != key && !t_held)
            acc += (unsigned __int128)((__int128)sre * sre) + (unsigned __int128)((__int128)sim * sim);
    }
    if (acc) add_u128(out, acc);
}

// Pack host-uploaded (key, re, im) arrays into records of one slot and check
// them: keys ascending within each vector, below 2^(2n), values nonzero and not
// -2^31.  A violation sets *bad (the caller rejects the call).
__global__ void k_pack_records(const uint64_t* __restrict__ keys, const int32_t* __restrict__ re,
                               const int32_t* __restrict__ im, const int64_t* __restrict__ off, int nseg,
                               const SegInfo* __restrict__ seginfo, Rec* __restrict__ dst, int* bad)
{
    const int64_t K = off[nseg];
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < K; i += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t key = keys[i];
        const int32_t a = re[i], b = im[i];
        const int s = seg_of(off, nseg, i);
        const int n = seginfo[s].n;
        const uint64_t lim = n == 32 ? ~0ull : ((1ull << (2 * n)) - 1ull);
        bool ok = (key & ~lim) == 0 && (a != 0 || b != 0) && a != INT32_MIN && b != INT32_MIN;
        if (ok && i > 0 && keys[i - 1] >= key && off[s] != i) ok = false;   // sorted inside each vector
        if (!ok) atomicExch(bad, 1);
        dst[i] = Rec{key, a, b};
    }
}

} // namespace

void launch_pack(const uint64_t* keys, const int32_t* re, const int32_t* im, const int64_t* off, int nseg,
                 const SegInfo* seginfo, Rec* dst, int* bad, cudaStream_t stream)
{
    k_pack_records<<<g_grid_misc ? g_grid_misc : 304, kThreads, 0, stream>>>(keys, re, im, off, nseg, seginfo, dst,
                                                                             bad);
}

void launch_obs(const StepParams& P, int which, SegStats* out, int grid, cudaStream_t stream)
{
    cudaMemsetAsync(out, 0, sizeof(SegStats) * P.nseg, stream);
    if (g_grid_misc == 0) configure_kernels();
    k_obs<<<grid > 0 && grid < g_grid_misc ? grid : g_grid_misc, kThreads, 0, stream>>>(P, which, out);
}

void launch_lookup(const StepParams& P, int seg, const uint64_t* q, int nq, int64_t* out, cudaStream_t stream)
{
    k_lookup<<<(nq + kThreads - 1) / kThreads, kThreads, 0, stream>>>(P, seg, q, nq, out);
}

const char* const kKernelNames[kNumTimedKernels] = {
    "k_prologue",     "k_spawn_draw",  "k_spawn_choose", "k_spawn_heavy", "k_bucket_hist",
    "k_bucket_scan",  "k_bucket_scatter", "k_bucket_sort", "k_sort_hist",  "k_sort_scatter",
    "k_spawn_segoff", "k_merge_plan",  "k_merge_part",   "k_merge",       "k_finalize"};

namespace {
// persistent grids: resident CTAs per SM x SMs, per kernel
int g_grid_spawn = 0, g_grid_choose = 0, g_grid_learned = 0, g_grid_heavy = 0, g_grid_heavy_learned = 0, g_grid_bsmall = 0, g_grid_bbig = 0, g_grid_sort = 0, g_grid_merge = 0, g_grid_learned_tc = 0;

int resident(const void* fn, int smem, int sms, int threads = kThreads)
{
    int per = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, fn, threads, smem) != cudaSuccess || per < 1) per = 1;
    return per * sms;
}
} // namespace

namespace {

// ---------------------------------------------------------------------------
// The learned proposal's integer weights Q_k for given sources under one
// program (a host query and the tests' handle on the forward pass): out[i *
// cap + k] for slot k of source i, 0 on slots of width 0.  FP32 network: one
// thread per source, the light kernel's arithmetic; tensor cores: one warp
// per 16 sources, the light kernel's forward pass and row weights.
// ---------------------------------------------------------------------------
__global__ void k_learned_weights(StepParams P, const uint8_t* __restrict__ pb, double t,
                                  const uint64_t* __restrict__ xs, const uint64_t* __restrict__ ys, int count,
                                  int64_t* __restrict__ out, int cap)
{
    const Prog prog = prog_at(pb);
    const LpNet net = lp_net(P);
    const int ns = prog.h->n_stat;
    const int64_t p_att = prog.h->p_att;
    const int n = P.n;
    const float tf32 = __double2float_rn(t);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < count; i += gridDim.x * blockDim.x) {
        const uint32_t x = (uint32_t)xs[i], y = (uint32_t)ys[i];
        float h1[kMaxHidden], h2[kMaxHidden];
        for (int q = 0; q < net.H; ++q) h1[q] = lp_h1(net, q, x, y, n, tf32);
        for (int q = 0; q < net.H; ++q) h2[q] = lp_h2(net, q, h1);
        float e[kMaxLearnedSlots];
        int16_t g[kMaxLearnedSlots];
        float m = -INFINITY;
        for (int k = 0; k < ns; ++k) {
            g[k] = (int16_t)(slot_width(prog, k) > 0 ? lp_output(P, prog.stat[k].mask) : -1);
            if (g[k] >= 0) {
                e[k] = lp_logit(net, g[k], h2);
                if (e[k] > m) m = e[k];
            }
        }
        float S = 0.0f;
        for (int k = 0; k < ns; ++k)
            if (g[k] >= 0) {
                e[k] = lp_exp(__fsub_rn(e[k], m));
                S = __fadd_rn(S, e[k]);
            }
        int64_t sum = 0, qa = -1;
        int arg = -1;
        for (int k = 0; k < ns; ++k) {
            const int64_t w = slot_width(prog, k);
            if (w <= 0) continue;
            const int64_t Q = lp_q(e[k], g[k] >= 0, S, P.mlp_eps, w, p_att);
            sum += Q;
            if (arg < 0 || Q > qa) {
                arg = k;
                qa = Q;
            }
        }
        for (int k = 0; k < ns; ++k) {
            const int64_t w = slot_width(prog, k);
            int64_t Q = w <= 0 ? 0 : lp_q(e[k], g[k] >= 0, S, P.mlp_eps, w, p_att);
            if (k == arg) Q += (1ll << 24) - sum;
            out[(int64_t)i * cap + k] = Q;
        }
    }
}

__global__ void __launch_bounds__(32) k_learned_weights_tc(StepParams P, const uint8_t* __restrict__ pb, double t,
                                                           const uint64_t* __restrict__ xs,
                                                           const uint64_t* __restrict__ ys, int count,
                                                           int64_t* __restrict__ out, int cap)
{
    extern __shared__ __align__(16) uint8_t tsm[];
    const TcLayout L = tc_layout(P.mlp_in, P.mlp_hidden, P.mlp_out);
    const int lane = threadIdx.x & 31;
    for (int i = lane; i < L.bytes / 16; i += 32) ((uint4*)tsm)[i] = ((const uint4*)P.mlp_tc)[i];
    TcSlots* slots = (TcSlots*)(tsm + L.bytes);
    const int ldo = L.Gp + 4;
    float* lgt = (float*)(tsm + L.bytes + sizeof(TcSlots));
    const Prog prog = prog_at(pb);
    tc_slots_fill(P, prog, slots, lane, 32);
    __syncthreads();
    const int ns = prog.h->n_stat;
    const int n = P.n;
    const float tb = __bfloat162float(__float2bfloat16_rn(__double2float_rn(t)));
    for (int tile = blockIdx.x; tile * 16 < count; tile += gridDim.x) {
        const int i = tile * 16 + lane;
        uint32_t x = 0u, y = 0u;
        if (lane < 16 && i < count) {
            x = (uint32_t)xs[i];
            y = (uint32_t)ys[i];
        }
        const int ga = lane >> 2, gb = ga + 8;
        const uint32_t xa = __shfl_sync(kFull, x, ga), ya = __shfl_sync(kFull, y, ga);
        const uint32_t xb = __shfl_sync(kFull, x, gb), yb = __shfl_sync(kFull, y, gb);
        tc_forward(tsm, L, n, xa, ya, tb, xb, yb, tb, lgt, ldo, lane);
        __syncwarp();
        const int r = lane & 15, half = lane >> 4;
        const bool act = tile * 16 + r < count;
        float* rlg = lgt + r * ldo;
        const TcRow tr = tc_pair_prepare(rlg, slots, ns, ns, P.mlp_eps, act, half);
        __syncwarp();
        if (half == 0 && act)
            for (int k = 0; k < ns; ++k) {
                int64_t Q = 0;
                if (slots->out[k] != -2) Q = tc_q(rlg, slots, k, tr.c) + (k == tr.arg ? tr.rem : 0);
                out[(int64_t)(tile * 16 + r) * cap + k] = Q;
            }
        __syncwarp();
    }
}

} // namespace

int learned_weights_smem(const StepParams& P)
{
    const TcLayout L = tc_layout(P.mlp_in, P.mlp_hidden, P.mlp_out);
    return L.bytes + (int)sizeof(TcSlots) + 16 * (L.Gp + 4) * 4;
}

void launch_learned_weights(const StepParams& P, bool tc, const uint8_t* prog, double t, const uint64_t* xs,
                            const uint64_t* ys, int count, int64_t* out, int cap, cudaStream_t stream)
{
    if (count <= 0) return;
    if (tc) {
        const int smem = learned_weights_smem(P);
        cudaFuncSetAttribute(k_learned_weights_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        k_learned_weights_tc<<<(count + 15) / 16, 32, smem, stream>>>(P, prog, t, xs, ys, count, out, cap);
    } else {
        k_learned_weights<<<(count + 127) / 128, 128, 0, stream>>>(P, prog, t, xs, ys, count, out, cap);
    }
}

void configure_kernels()
{
    cudaFuncSetAttribute(k_merge, cudaFuncAttributeMaxDynamicSharedMemorySize, kMergeSmem);
    cudaFuncSetAttribute(k_spawn_draw, cudaFuncAttributeMaxDynamicSharedMemorySize, kDrawSmem);
    cudaFuncSetAttribute(k_bucket_sort_big, cudaFuncAttributeMaxDynamicSharedMemorySize, kBigSortSmem);
    int dev = 0, sms = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    g_grid_spawn = resident((const void*)k_spawn_draw, kDrawSmem, sms);
    g_grid_choose = resident((const void*)k_spawn_choose, 0, sms);
    g_grid_learned = resident((const void*)k_spawn_learned, 0, sms);
    g_grid_heavy = resident((const void*)k_spawn_heavy, 0, sms);
    g_grid_heavy_learned = resident((const void*)k_spawn_heavy_learned, 0, sms);
    g_grid_sort = resident((const void*)k_sort_scatter, 0, sms);
    g_grid_merge = resident((const void*)k_merge, kMergeSmem, sms, kMergeThreads);
    g_grid_bsmall = resident((const void*)k_bucket_sort_small, 0, sms);
    g_grid_bbig = resident((const void*)k_bucket_sort_big, kBigSortSmem, sms);
    g_grid_misc = 2 * sms;
    // tensor-core proposal: sized for the largest network (64 hidden, 256 outputs, 80 inputs)
    const TcLayout big = tc_layout(kTcMaxIp, kTcMaxH, kTcMaxGp);
    const int tc_light = tc_smem_bytes(big, kTcWarps);
    const int tc_heavy = big.bytes + (int)sizeof(TcSlots) + 16 * (big.Gp + 4) * 4;
    cudaFuncSetAttribute(k_spawn_learned_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, tc_light);
    cudaFuncSetAttribute(k_spawn_heavy_learned_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, tc_heavy);
    g_grid_learned_tc = resident((const void*)k_spawn_learned_tc, tc_light, sms, kTcWarps * 32);
}

// Persistent grid of the tensor-core proposal's light kernel for its actual
// shared memory (the network's size sets it).
int tc_grid(int smem)
{
    static int cached_smem = -1, cached_grid = 0;
    if (smem != cached_smem) {
        int dev = 0, sms = 1;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cached_grid = resident((const void*)k_spawn_learned_tc, smem, sms, kTcWarps * 32);
        cached_smem = smem;
    }
    return cached_grid;
}

void launch_step(const StepParams& P, int grid, cudaStream_t stream, cudaEvent_t* ev)
{
    if (g_grid_spawn == 0) configure_kernels();
    // grid > 0 caps every persistent or grid-stride kernel at that many CTAs
    auto cap = [grid](int g) { return grid > 0 && grid < g ? grid : g; };
    // ev (optional): kNumTimedKernels + 1 events; kernel i runs between ev[i] and ev[i + 1]
    auto mark = [&](int i) { if (ev) cudaEventRecord(ev[i], stream); };
    mark(0);
    k_prologue<<<1, kThreads, 0, stream>>>(P);
    mark(1);
    k_spawn_draw<<<cap(g_grid_spawn), kThreads, kDrawSmem, stream>>>(P);
    mark(2);
    const TcLayout TL = tc_layout(P.mlp_in, P.mlp_hidden, P.mlp_out);
    if (P.proposal == 2)   // timed in the choose slot
        k_spawn_learned<<<cap(g_grid_learned), kThreads, 0, stream>>>(P);
    else if (P.proposal == 3)
        k_spawn_learned_tc<<<cap(tc_grid(tc_smem_bytes(TL, kTcWarps))), kTcWarps * 32, tc_smem_bytes(TL, kTcWarps),
                             stream>>>(P);
    else
        k_spawn_choose<<<cap(g_grid_choose), kThreads, 0, stream>>>(P);
    mark(3);
    if (P.proposal == 2)
        k_spawn_heavy_learned<<<cap(g_grid_heavy_learned), kThreads, 0, stream>>>(P);
    else if (P.proposal == 3)
        k_spawn_heavy_learned_tc<<<cap(g_grid_heavy_learned), kThreads,
                                   TL.bytes + (int)sizeof(TcSlots) + 16 * (TL.Gp + 4) * 4, stream>>>(P);
    else
        k_spawn_heavy<<<cap(g_grid_heavy), kThreads, 0, stream>>>(P);
    mark(4);
    if (P.sort_mode) {
        k_bucket_hist<<<cap(g_grid_misc), kThreads, 0, stream>>>(P);
        mark(5);
        k_bucket_scan<<<((1 << P.bucket_bits) + 1023) / 1024, 1024, 0, stream>>>(P);
        mark(6);
        k_bucket_scatter<<<cap(g_grid_misc), kThreads, 0, stream>>>(P);
        mark(7);
        if (P.sort_mode == 1) {
            k_bucket_sort_small<<<cap(g_grid_bsmall), kThreads, 0, stream>>>(P);
            k_bucket_sort_big<<<cap(g_grid_bbig), kThreads, kBigSortSmem, stream>>>(P);
        }
        mark(8);
    } else {
        mark(5);
        mark(6);
        mark(7);
        mark(8);
    }
    // LSD radix sort: every pass returns at once unless the step sorts this way
    const int np = P.key_passes + P.seg_passes;
    k_sort_hist<<<cap(g_grid_misc), kThreads, 0, stream>>>(P);
    mark(9);
    SRec* a = P.spawn;
    SRec* b = P.spawn_alt;
    for (int p = 0; p < np; ++p) {
        k_sort_scatter<<<cap(g_grid_sort), kThreads, 0, stream>>>(P, p, a, b);
        SRec* t = a;
        a = b;
        b = t;
    }
    mark(10);
    k_spawn_segoff<<<(P.nseg + 1 + kThreads - 1) / kThreads, kThreads, 0, stream>>>(P);
    mark(11);
    k_merge_plan<<<1, 1024, 0, stream>>>(P);
    mark(12);
    k_merge_part<<<cap(g_grid_misc), kThreads, 0, stream>>>(P);
    mark(13);
    k_merge<<<cap(g_grid_merge), kMergeThreads, kMergeSmem, stream>>>(P);
    mark(14);
    k_finalize<<<1, 1024, 0, stream>>>(P);
    mark(15);
}

int step_launch_count(const StepParams& P)
{
    const int np = P.key_passes + P.seg_passes;
    const int bucket = P.sort_mode == 0 ? 0 : (P.sort_mode == 1 ? 5 : 3);
    // prologue, draw, choose, heavy; bucket sort; LSD histogram and passes;
    // segment offsets, merge plan, partition, merge, finalize
    return 4 + bucket + 1 + np + 5;
}

void launch_overlap_all(const StepParams& P, const uint64_t* idx, const double* psi, int len, double* out,
                        cudaStream_t stream)
{
    k_overlap_all<<<P.nseg, kThreads, 0, stream>>>(P, idx, psi, len, out);
}

void launch_antiherm(const StepParams& P, unsigned long long* out, int grid, cudaStream_t stream)
{
    if (g_grid_spawn == 0) configure_kernels();
    cudaMemsetAsync(out, 0, (size_t)P.nseg * 16, stream);
    k_antiherm<<<grid > 0 ? grid : g_grid_misc, kThreads, 0, stream>>>(P, out);
}

// The packed fp32 parameters in the tensor-core layout: one thread per
// element of the padded buffer (weights rounded to bf16, padding zero).
__global__ void k_mlp_tc_pack(const float* __restrict__ prm, TcLayout L, uint8_t* __restrict__ out)
{
    const int I = L.I, H = L.H, G = L.G;
    const float* w1 = prm;
    const float* b1 = w1 + H * I;
    const float* w2 = b1 + H;
    const float* b2 = w2 + H * H;
    const float* w3 = b2 + H;
    const float* b3 = w3 + G * H;
    const int n1 = H * L.ld1, n2 = H * L.ld2, n3 = L.Gp * L.ld3;
    const int total = n1 + n2 + n3 + 2 * H + L.Gp;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < total; e += gridDim.x * blockDim.x) {
        if (e < n1) {
            const int r = e / L.ld1, c = e % L.ld1;
            ((__nv_bfloat16*)(out + L.o_w1))[e] = __float2bfloat16_rn(c < I ? w1[r * I + c] : 0.0f);
        } else if (e < n1 + n2) {
            const int f = e - n1, r = f / L.ld2, c = f % L.ld2;
            ((__nv_bfloat16*)(out + L.o_w2))[f] = __float2bfloat16_rn(c < H ? w2[r * H + c] : 0.0f);
        } else if (e < n1 + n2 + n3) {
            const int f = e - n1 - n2, r = f / L.ld3, c = f % L.ld3;
            ((__nv_bfloat16*)(out + L.o_w3))[f] = __float2bfloat16_rn(c < H && r < G ? w3[r * H + c] : 0.0f);
        } else {
            const int f = e - n1 - n2 - n3;
            if (f < H) ((float*)(out + L.o_b1))[f] = b1[f];
            else if (f < 2 * H) ((float*)(out + L.o_b2))[f - H] = b2[f - H];
            else ((float*)(out + L.o_b3))[f - 2 * H] = (f - 2 * H) < G ? b3[f - 2 * H] : 0.0f;
        }
    }
}

void launch_mlp_tc_pack(const float* params, const TcLayout& L, uint8_t* out, cudaStream_t stream)
{
    cudaMemsetAsync(out, 0, (size_t)L.bytes, stream);
    k_mlp_tc_pack<<<64, 256, 0, stream>>>(params, L, out);
}

void launch_antiherm_sum(const StepParams& P, const int32_t* segs, int count, unsigned long long* out, int grid,
                         cudaStream_t stream)
{
    if (g_grid_spawn == 0) configure_kernels();
    cudaMemsetAsync(out, 0, 16, stream);
    const int gx = grid > 0 ? grid : (g_grid_misc + count - 1) / count;
    k_antiherm_sum<<<dim3(gx > 0 ? gx : 1, count), kThreads, 0, stream>>>(P, segs, count, out);
}

void launch_init(const StepParams& P, const uint64_t* x, const uint64_t* y, const double* re, const double* im,
                 int64_t nnz, int64_t* tmp_vals, cudaStream_t stream)
{
    const int64_t total = nnz * P.nseg;
    const int blocks = (int)((total + kThreads - 1) / kThreads < 4096 ? (total + kThreads - 1) / kThreads : 4096);
    k_init_values<<<blocks > 0 ? blocks : 1, kThreads, 0, stream>>>(P, x, y, re, im, nnz, tmp_vals);
    k_init_compact<<<1, kThreads, 0, stream>>>(P, x, y, nnz, tmp_vals);
}

} // namespace qmc
