// The step for 33..60 qubits, where a key (x << n) | y needs 128 bits
// (arXiv:2502.18929: the method of the 64-bit step, same random stream).
//
//   k_wide_prologue     per-step Philox keys, counter resets
//   k_wide_abound       where each bucket of the spawn sort starts in N(t)
//   k_wide_spawn        spawning [End Matter, spawn step] of parents with few
//                       walkers: one thread per rank group of four parents,
//                       walkers that pass the prefilter become candidates
//   k_wide_choose       candidates: exact column weight, full draw, spawn record
//   k_wide_heavy        one CTA per chunk of a heavy parent's walkers, the
//                       column laid out once as bins of the draw
//   k_wide_bhist ..
//   k_wide_bsort_big    bucket sort of the spawns by (vector, key): bucket
//                       counts, their prefix, one counting pass, windows of
//                       whole buckets sorted in shared memory
//   k_wide_hist         (LSD fallback when a bucket is too large) digit counts
//                       of every 8-bit radix pass of (vector, key)
//   k_wide_plan         passes to skip (a digit shared by every record) and
//                       the ping-pong buffer of each pass
//   k_wide_tile_hist /
//   k_wide_tile_scan /
//   k_wide_scatter      one stable LSD pass: per-tile counts, their prefix
//                       over tiles per digit, scatter with warp-match ranks
//   k_wide_spawn_off    vector boundaries of the sorted spawns
//   k_wide_runs         runs of equal keys: summed spawns under the initiator
//                       rule, the key's position in N(t), per merge tile the
//                       records zeroed and the new keys
//   k_wide_mtop         survivors and new keys before every merge tile
//   k_wide_scan_*       exclusive prefix sums of the new keys
//   k_wide_merge_a /
//   k_wide_scatter_u    N(t + dt) = the survivors in key order [End Matter,
//                       annihilation step], with the per-vector observables
//   k_wide_outoff       vector offsets of N(t + dt)
//   k_wide_finalize     history, counters, rotate the slots
//
// Integer-only, like the 64-bit step: results are bit-identical to the
// oracle whatever the launch shape.
#include <cuda_runtime.h>
#include <stdint.h>

#include "column_eval.h"
#include "device_common.h"
#include "kernels.h"
#include "wide.h"

namespace qmc {

namespace {

constexpr int kWThreads = 256;

__device__ __forceinline__ u128 wkey(uint64_t lo, uint64_t hi) { return ((u128)hi << 64) | (u128)lo; }
__device__ __forceinline__ u128 wkey(const WRec& r) { return wkey(r.lo, r.hi); }
__device__ __forceinline__ u128 wkey(const WSpawn& r) { return wkey(r.lo, r.hi); }

// A population slot in structure-of-arrays form: pop_cap 16-byte keys (low
// word, high word), then pop_cap 8-byte values (re, im) -- 24 bytes a record,
// keys and values each read with one vector access.
struct WPop {
    ulonglong2* key;
    int2* val;
};

__device__ __forceinline__ WPop wpop(const StepParams& P, int slot)
{
    uint8_t* b = (uint8_t*)P.pop[slot];
    return WPop{(ulonglong2*)b, (int2*)(b + 16 * P.pop_cap)};
}

__device__ __forceinline__ u128 wkey(const ulonglong2& k) { return ((u128)k.y << 64) | (u128)k.x; }

__device__ __forceinline__ WRec wload(const WPop& p, int64_t i)
{
    const ulonglong2 k = __ldg(&p.key[i]);
    const int2 v = __ldg(&p.val[i]);
    WRec r;
    r.lo = k.x;
    r.hi = k.y;
    r.re = v.x;
    r.im = v.y;
    return r;
}

__device__ __forceinline__ void wstore(const WPop& p, int64_t i, u128 key, int32_t re, int32_t im)
{
    p.key[i] = make_ulonglong2((unsigned long long)(uint64_t)key, (unsigned long long)(uint64_t)(key >> 64));
    p.val[i] = make_int2(re, im);
}

__device__ __forceinline__ WSpawn wsload(const WSpawn* p, int64_t i)
{
    WSpawn r;
    r.lo = p[i].lo;
    r.hi = p[i].hi;
    r.meta = p[i].meta;
    r.val = p[i].val;
    return r;
}

__device__ __forceinline__ uint32_t lanemask_lt()
{
    uint32_t m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// Program of one instance for one pass of the current step.
__device__ __forceinline__ const uint8_t* prog_of(const StepParams& P, const StepInfo& inf, int inst, int phase)
{
    const int64_t* tab = (const int64_t*)(P.progs + inf.tab_off);
    return P.progs + tab[2 * inst + phase];
}

// The spawn record of a walker of component comp (0 real, 1 imaginary) whose
// parent's value has sign sg there, onto dest through channel chan of an
// element of sign v, with the paper's sign rule [End Matter, spawn step]: the
// Re channel keeps the component, the Im channel multiplies by i; sigma = -1
// for the N(t - dt) pass.
__device__ __forceinline__ WSpawn wide_record(u128 dest, int seg, int comp, int chan, int64_t v, int sg, int phase,
                                              int noninit)
{
    const int s = (phase ? -1 : 1) * sg * (v > 0 ? 1 : -1);
    int target, val;
    if (chan == 0) { target = comp; val = s; }
    else if (comp == 0) { target = 1; val = s; }
    else { target = 0; val = -s; }
    WSpawn r;
    r.lo = (uint64_t)dest;
    r.hi = (uint64_t)(dest >> 64);
    r.meta = ((uint32_t)seg << 2) | ((uint32_t)target << 1) | (uint32_t)noninit;
    r.val = val;
    return r;
}

// Records a warp appends to a global array (dst, capacity cap, counter
// total), gathered in kCap slots of shared memory: one atomic on the counter
// and one contiguous copy per full stage instead of one atomic per round.
// Every call is made by all 32 lanes; count is the same in every lane.
template <typename T, int kCap>
struct WarpStage {
    T* buf;
    int count;

    __device__ __forceinline__ void flush(unsigned long long* total, T* dst, int64_t cap, DevState* st,
                                          uint32_t err, int lane)
    {
        __syncwarp();
        if (count == 0) return;
        unsigned long long b = 0;
        if (lane == 0) b = atomicAdd(total, (unsigned long long)count);
        b = __shfl_sync(kFull, b, 0);
        for (int j = lane; j < count; j += 32) {
            const int64_t pos = (int64_t)b + j;
            if (pos < cap) dst[pos] = buf[j];
            else set_error(st, err);
        }
        __syncwarp();
        count = 0;
    }

    __device__ __forceinline__ void push(bool on, const T& v, unsigned long long* total, T* dst, int64_t cap,
                                         DevState* st, uint32_t err, int lane)
    {
        const uint32_t bal = __ballot_sync(kFull, on);
        if (!bal) return;
        const int n = __popc(bal);
        if (count + n > kCap) flush(total, dst, cap, st, err, lane);
        if (on) buf[count + __popc(bal & lanemask_lt())] = v;
        count += n;
    }
};

constexpr int kWStage = 128;   // staged records per warp

// Append the spawns the lanes of a warp hold (sp) with one atomic.
__device__ __forceinline__ void warp_append(const StepParams& P, const WideParams& W, bool sp, const WSpawn& rec,
                                            int lane)
{
    const uint32_t bal = __ballot_sync(kFull, sp);
    if (!bal) return;
    const int leader = __ffs(bal) - 1;
    unsigned long long base = 0;
    if (lane == leader) base = atomicAdd((unsigned long long*)&P.st->spawn_total, (unsigned long long)__popc(bal));
    base = __shfl_sync(kFull, base, leader);
    if (sp) {
        const int64_t pos = (int64_t)base + __popc(bal & lanemask_lt());
        if (pos < P.spawn_cap) W.spawn[pos] = rec;
        else set_error(P.st, DERR_SPAWN_CAPACITY);
    }
}

} // namespace

namespace {

// ---------------------------------------------------------------------------
// Prologue (single CTA): keys of this step, counter resets.
// ---------------------------------------------------------------------------
__global__ void k_wide_prologue(StepParams P)
{
    DevState* st = P.st;
    if (read_error(st)) return;
    const uint64_t step = st->step;
    for (int s = threadIdx.x; s < P.nseg; s += blockDim.x) {
        const SegInfo si = P.seginfo[s];
        const uint64_t seed = P.inst[si.inst].seed;
        const uint4 o = philox10(make_uint4((uint32_t)step, (uint32_t)(step >> 32), (uint32_t)si.vec, kTagStep),
                                 make_uint2((uint32_t)seed, (uint32_t)(seed >> 32)));
        P.kd[s] = make_uint2(o.x, o.y);
        P.segacc[s] = SegStats{0ull, 0ll, 0ll, 0ll};
    }
    // rank-group offsets of N(t) and N(t - dt) (the light spawn's work
    // units): gof[s] = sum over the vectors before s of ceil(K / 4)
    __shared__ long long wsum[kWThreads / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int w = 0; w < 2; ++w) {
        const int slot = w ? (st->cur + 2) % 3 : st->cur;
        const int64_t* off = P.segoff[slot];
        int64_t* gof = P.gofs[slot];
        long long carry = 0;
        for (int base = 0; base < P.nseg; base += kWThreads) {
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
            for (int q = 0; q < kWThreads / 32; ++q) {
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
        st->heavy_total = 0;
        st->next_total = 0;
        st->merge_tiles = 0;
        st->sort_fallback = P.sort_mode == 0 ? 1u : 0u;
    }
}

// ---------------------------------------------------------------------------
// Spawning of light parents: one thread per rank group of four consecutive
// parents of a vector, so that one Philox call gives the 32-bit words of the
// group's first walkers (a second call their second walkers); the warp's
// lanes step through their walkers together so that each round's spawns take
// one atomic.  A walker's exact draw and the parent's column weight are
// evaluated only when its word passes the program's prefilter.  A parent with
// more than kWLight walkers becomes heavy work items.
// ---------------------------------------------------------------------------
__device__ __forceinline__ int wgroup_seg(const int64_t* gof, int nseg, int64_t g)
{
    int lo = 0, hi = nseg - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (__ldg(&gof[mid]) <= g) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// Candidate record (four words): parent index in its slot, vector, the
// walker's 32-bit word W, and cand_word: the walker's index j in its
// component (20 bits), the component, the pass, the initiator flag and the
// sign of the parent's value in that component (bits 20 .. 23).
constexpr uint32_t kWJ20 = (1u << 20) - 1u;

__device__ __forceinline__ uint32_t cand_word(int64_t w, int32_t re, int32_t im, int phase, int non)
{
    const int64_t are = iabs64(re);
    const int comp = w < are ? 0 : 1;
    const uint32_t j = (uint32_t)(comp ? w - are : w);
    const int pos = comp ? (im > 0) : (re > 0);
    return j | ((uint32_t)comp << 20) | ((uint32_t)phase << 21) | ((uint32_t)non << 22) | ((uint32_t)pos << 23);
}

__global__ void __launch_bounds__(kWThreads) k_wide_spawn(StepParams P, WideParams W, int phase)
{
    __shared__ uint4 s_cand[kWThreads / 32][kWStage];
    DevState* st = P.st;
    if (cta_error(st)) return;
    if (phase == 0 && P.sort_mode != 0)   // bucket counters of this step's spawn sort
        for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < (1 << P.bucket_bits); b += gridDim.x * blockDim.x)
            P.bucket[b] = 0u;
    const StepInfo inf = P.info[st->call_index];
    if (phase == 1 && !inf.ab2) return;
    const int slot = phase ? (st->cur + 2) % 3 : st->cur;
    const WPop pop = wpop(P, slot);
    const int64_t* off = P.segoff[slot];
    const int64_t* gof = P.gofs[slot];
    const int64_t G = gof[P.nseg];
    const int lane = threadIdx.x & 31;
    WarpStage<uint4, kWStage> cs{s_cand[threadIdx.x >> 5], 0};
    unsigned long long* ctot = (unsigned long long*)&st->cand_total;
    uint4* cdst = (uint4*)P.cand;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31); base < G; base += stride) {
        const int64_t g = base + lane;
        int64_t m[4] = {0, 0, 0, 0};
        int32_t vre[4] = {0, 0, 0, 0}, vim[4] = {0, 0, 0, 0};
        int non[4] = {0, 0, 0, 0};
        int seg = 0;
        uint32_t grp = 0;
        int64_t first = 0;
        uint2 kd = make_uint2(0u, 0u);
        int64_t pre = -1;
        // the vector of the warp's first group with its prefilter bound and
        // key, then per lane only across a boundary
        int seg0 = 0;
        int64_t pre0 = 0, imin0 = 0;
        uint2 kd0 = make_uint2(0u, 0u);
        if (lane == 0) {
            seg0 = wgroup_seg(gof, P.nseg, base);
            const int in0 = P.seginfo[seg0].inst;
            pre0 = wprog_at(prog_of(P, inf, in0, phase)).h->p_bound >> 20;
            imin0 = P.inst[in0].init_min;
            kd0 = P.kd[seg0];
        }
        seg0 = __shfl_sync(kFull, seg0, 0);
        pre0 = __shfl_sync(kFull, pre0, 0);
        imin0 = __shfl_sync(kFull, imin0, 0);
        kd0.x = __shfl_sync(kFull, kd0.x, 0);
        kd0.y = __shfl_sync(kFull, kd0.y, 0);
        const int64_t seg0_end = gof[seg0 + 1];
        if (g < G) {
            seg = g < seg0_end ? seg0 : wgroup_seg(gof, P.nseg, g);
            grp = (uint32_t)(g - gof[seg]);
            first = off[seg] + 4 * (int64_t)grp;
            const int cnt = (int)min((int64_t)4, off[seg + 1] - first);
            kd = seg == seg0 ? kd0 : P.kd[seg];
            pre = seg == seg0 ? pre0 : wprog_at(prog_of(P, inf, P.seginfo[seg].inst, phase)).h->p_bound >> 20;
            const int64_t imin = seg == seg0 ? imin0 : P.inst[P.seginfo[seg].inst].init_min;
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                if (k >= cnt) break;
                const int2 v = __ldg(&pop.val[first + k]);
                m[k] = iabs64(v.x) + iabs64(v.y);
                vre[k] = v.x;
                vim[k] = v.y;
                non[k] = (imin > 0 && m[k] < imin) ? 1 : 0;
                if (m[k] > kWLight) {
                    const int64_t nb = (m[k] - 2 + 3) / 4;
                    const int64_t chunks = (nb + kWChunk - 1) / kWChunk;
                    const int64_t at =
                        (int64_t)atomicAdd((unsigned long long*)&st->heavy_total, (unsigned long long)chunks);
                    for (int64_t c = 0; c < chunks; ++c) {
                        if (at + c < P.heavy_cap)
                            P.heavy[at + c] = HeavyItem{first + k, phase, 0, (int32_t)c, seg};
                        else
                            set_error(st, DERR_HEAVY_CAPACITY);
                    }
                    m[k] = 0;
                }
            }
        }
        // first walkers: one call for the group; the candidates go through
        // the warp's stage
        const uint4 gw0 = g < G ? group_words(grp, 0u, phase, kd) : make_uint4(0u, 0u, 0u, 0u);
#pragma unroll
        for (int k = 0; k < 4; ++k)
            cs.push(m[k] > 0 && (int64_t)word_of(gw0, k) <= pre,
                    make_uint4((uint32_t)(first + k), (uint32_t)seg, word_of(gw0, k),
                               cand_word(0, vre[k], vim[k], phase, non[k])),
                    ctot, cdst, P.cand_cap, st, DERR_CAND_CAPACITY, lane);
        // second walkers: one more call; further walkers: the parent's calls
        const bool two = m[0] > 1 || m[1] > 1 || m[2] > 1 || m[3] > 1;
        if (__any_sync(kFull, two)) {
            const uint4 gw1 = two ? group_words(grp, 1u, phase, kd) : make_uint4(0u, 0u, 0u, 0u);
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const uint32_t rank = 4u * grp + (uint32_t)k;
                const int64_t mk = m[k];
                for (int64_t w = 1; __any_sync(kFull, w < mk); ++w) {
                    uint32_t Wd = 0u;
                    if (w < mk)
                        Wd = w == 1 ? word_of(gw1, k)
                                    : word_of(extra_words(rank, (uint32_t)((w - 2) >> 2), phase, kd), (int)((w - 2) & 3));
                    const bool on = w < mk && (int64_t)Wd <= pre;
                    cs.push(on,
                            make_uint4((uint32_t)(first + k), (uint32_t)seg, Wd,
                                       cand_word(w, vre[k], vim[k], phase, non[k])),
                            ctot, cdst, P.cand_cap, st, DERR_CAND_CAPACITY, lane);
                }
            }
        }
    }
    cs.flush(ctot, cdst, P.cand_cap, st, DERR_CAND_CAPACITY, lane);
}

// Candidates: the parent's exact column weight, the walker's full draw and,
// if it spawns, its record.
__global__ void __launch_bounds__(kWThreads, 3) k_wide_choose(StepParams P, WideParams W)
{
    __shared__ WSpawn s_sp[kWThreads / 32][kWStage];
    DevState* st = P.st;
    if (cta_error(st)) return;
    const StepInfo inf = P.info[st->call_index];
    const int64_t total = min((int64_t)st->cand_total, P.cand_cap);
    const int lane = threadIdx.x & 31;
    WarpStage<WSpawn, kWStage> ss{s_sp[threadIdx.x >> 5], 0};
    unsigned long long* stot = (unsigned long long*)&st->spawn_total;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31); base < total; base += stride) {
        const int64_t i = base + lane;
        WSpawn sr;
        bool sp = false;
        if (i < total) {
            const uint4 c = ((const uint4*)P.cand)[i];
            const int comp = (int)((c.w >> 20) & 1u), phase = (int)((c.w >> 21) & 1u);
            const int non = (int)((c.w >> 22) & 1u), sg = ((c.w >> 23) & 1u) ? 1 : -1;
            const int slot = phase ? (st->cur + 2) % 3 : st->cur;
            const int seg = (int)c.y;
            const uint32_t rank = c.x - (uint32_t)__ldg(&P.segoff[slot][seg]);
            const SegInfo si = P.seginfo[seg];
            const u128 key = wkey(__ldg(&wpop(P, slot).key[c.x]));
            const uint64_t x = (uint64_t)(key >> si.n), y = (uint64_t)key & ((1ull << si.n) - 1ull);
            const WProg pr = wprog_at(prog_of(P, inf, si.inst, phase));
            int64_t sre, sim;
            const int64_t Pw = column_weight(pr, x, y, &sre, &sim);
            if (Pw >= (1ll << 52)) {
                set_error(st, DERR_DT_TOO_LARGE);
            } else if ((int64_t)c.z <= ((Pw - 1) >> 20)) {
                // the walker's full draw T = W << 20 | L [reading R3]
                const int64_t T = walker_T(c.z, rank, c.w & kWJ20, comp, phase, P.kd[seg]);
                u128 mask;
                int chan;
                int64_t v;
                if (T < Pw && choose_destination(pr, x, y, sre, sim, T, &mask, &chan, &v)) {
                    sp = true;
                    sr = wide_record(key ^ mask, seg, comp, chan, v, sg, phase, non);
                }
            }
        }
        ss.push(sp, sr, stot, W.spawn, P.spawn_cap, st, DERR_SPAWN_CAPACITY, lane);
    }
    ss.flush(stot, W.spawn, P.spawn_cap, st, DERR_SPAWN_CAPACITY, lane);
}

// ---------------------------------------------------------------------------
// Heavy parents: one CTA per work item.  Item c of a parent covers the
// walkers 2 + 4 b + (0..3) of its extra calls b in [c kWChunk, (c + 1)
// kWChunk), item 0 also the walkers 0 and 1.  The parent's column is laid out
// once per item in shared memory: one thread evaluates its weight P and
// diagonal element, all threads the destination entries' elements, whose
// |Re| and |Im| in the canonical order are the bins of the walkers' draw T
// over [0, P) (the order choose_destination walks), with a table of the first
// bin of each 2^s-wide slice of [0, P).  A spawned walker finds its bin with
// one or two reads; the walkers are counted per (bin, walker component) and
// leave as one record per nonzero count (the merge adds records, so the
// populations are those of one record per walker).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kWThreads) k_wide_heavy(StepParams P, WideParams W)
{
    __shared__ int64_t cum[2 * kMaxEntries];   // bin widths, then their inclusive prefix
    __shared__ int hist[4 * kMaxEntries];      // spawned walkers per (bin, component)
    __shared__ int8_t sgnv[2 * kMaxEntries];   // sign of each bin's element
    __shared__ uint16_t sidx[1025];            // first bin of each slice of [0, P)
    __shared__ int64_t s_col[3];               // P and the diagonal element's Re, Im
    __shared__ int64_t warp_tot[kWThreads / 32];
    DevState* st = P.st;
    if (cta_error(st)) return;
    const StepInfo inf = P.info[st->call_index];
    const int64_t items = min((int64_t)st->heavy_total, P.heavy_cap);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (int e = tid; e < 4 * kMaxEntries; e += blockDim.x) hist[e] = 0;
    __syncthreads();
    for (int64_t it = blockIdx.x; it < items; it += gridDim.x) {
        const HeavyItem h = P.heavy[it];
        const int slot = h.phase ? (st->cur + 2) % 3 : st->cur;
        const int seg = h.seg;
        const SegInfo si = P.seginfo[seg];
        const WRec r = wload(wpop(P, slot), h.parent);
        const u128 key = wkey(r);
        const uint64_t x = (uint64_t)(key >> si.n), y = (uint64_t)key & ((1ull << si.n) - 1ull);
        const WProg pr = wprog_at(prog_of(P, inf, si.inst, h.phase));
        const int ne = pr.h->n_entry, nb = 2 * ne;
        if (tid == 0) {
            int64_t a, b;
            s_col[0] = column_weight(pr, x, y, &a, &b);
            s_col[1] = a;
            s_col[2] = b;
        }
        __syncthreads();
        const int64_t Pw = s_col[0];
        if (Pw >= (1ll << 52) || ne > kMaxEntries) {   // the same in every thread
            if (tid == 0) set_error(st, Pw >= (1ll << 52) ? DERR_DT_TOO_LARGE : DERR_TILE_CAPACITY);
            return;
        }
        for (int e = tid; e < ne; e += blockDim.x) {
            int64_t vr, vi;
            entry_value(pr, pr.ent[e], x, y, s_col[1], s_col[2], &vr, &vi);
            cum[2 * e] = iabs64(vr);
            cum[2 * e + 1] = iabs64(vi);
            sgnv[2 * e] = vr > 0 ? 1 : -1;
            sgnv[2 * e + 1] = vi > 0 ? 1 : -1;
        }
        __syncthreads();
        {   // inclusive prefix of the bin widths, in place (blocked per thread, then across threads)
            const int per = (nb + kWThreads - 1) / kWThreads;
            const int b0 = min(nb, tid * per), b1 = min(nb, b0 + per);
            int64_t acc = 0;
            for (int b = b0; b < b1; ++b) acc += cum[b];
            int64_t incl = acc;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int64_t t = __shfl_up_sync(kFull, incl, o);
                if (lane >= o) incl += t;
            }
            if (lane == 31) warp_tot[warp] = incl;
            __syncthreads();
            int64_t run = incl - acc;
            for (int q = 0; q < warp; ++q) run += warp_tot[q];
            for (int b = b0; b < b1; ++b) {
                run += cum[b];
                cum[b] = run;
            }
        }
        __syncthreads();
        // first bin of each 2^ish-wide slice of [0, P): about eight slices per bin, at most 1024
        int ish = 0;
        if (nb > 0) {
            const int64_t slices = nb < 128 ? 8 * nb : 1024;
            while ((Pw >> ish) >= slices) ++ish;
            const int nbk = (int)(Pw >> ish) + 1;
            for (int k = tid; k < nbk; k += blockDim.x) {
                const int64_t t0 = (int64_t)k << ish;
                int lo = 0, hi = nb - 1;
                while (lo < hi) {
                    const int mid = (lo + hi) >> 1;
                    if (cum[mid] > t0) hi = mid; else lo = mid + 1;
                }
                sidx[k] = (uint16_t)lo;
            }
        }
        __syncthreads();
        const int64_t are = iabs64(r.re), m = are + iabs64(r.im);
        const uint32_t rank = (uint32_t)(h.parent - P.segoff[slot][seg]);
        const uint2 kd = P.kd[seg];
        const int64_t pre = (Pw - 1) >> 20;
        // walker w with its 32-bit word W [reading R3]: the prefilter, the full
        // draw T = W << 20 | L, T < P, its bin
        auto walker = [&](int64_t w, uint32_t Wd) {
            if ((int64_t)Wd > pre) return;
            const int comp = w < are ? 0 : 1;
            const uint32_t j = (uint32_t)(comp ? w - are : w);
            const int64_t T = walker_T(Wd, rank, j, comp, h.phase, kd);
            if (T >= Pw) return;
            int lo = sidx[T >> ish];   // first bin with cum > T
            while (lo < nb - 1 && cum[lo] <= T) ++lo;
            atomicAdd(&hist[2 * lo + comp], 1);
        };
        if (h.chunk == 0 && tid < 2 && tid < m)
            walker(tid, word_of(group_words(rank >> 2, (uint32_t)tid, h.phase, kd), (int)(rank & 3u)));
        const int64_t ncall = (m - 2 + 3) / 4;
        const int64_t c0 = (int64_t)h.chunk * kWChunk, c1 = min(ncall, c0 + kWChunk);
        for (int64_t b = c0 + tid; b < c1; b += blockDim.x) {
            const uint4 o = extra_words(rank, (uint32_t)b, h.phase, kd);
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const int64_t w = 2 + 4 * b + k;
                if (w < m) walker(w, word_of(o, k));
            }
        }
        __syncthreads();
        // one record per nonzero count, in rounds of the block's threads
        const int64_t init_min = P.inst[si.inst].init_min;
        const int noninit = (init_min > 0 && m < init_min) ? 1 : 0;
        const int nslots = 2 * nb;
        for (int base = 0; base < nslots; base += blockDim.x) {
            const int idx = base + tid;
            WSpawn sr;
            bool sp = false;
            if (idx < nslots) {
                const int cnt = hist[idx];
                if (cnt) {
                    hist[idx] = 0;
                    const int bin = idx >> 1, comp = idx & 1;
                    const int sg = comp == 0 ? (r.re > 0 ? 1 : -1) : (r.im > 0 ? 1 : -1);
                    sr = wide_record(key ^ pr.ent[bin >> 1].mask_key, seg, comp, bin & 1, sgnv[bin], sg, h.phase,
                                     noninit);
                    sr.val *= cnt;
                    sp = true;
                }
            }
            warp_append(P, W, sp, sr, lane);
        }
        __syncthreads();
    }
}

} // namespace

namespace {

// ---------------------------------------------------------------------------
// LSD radix sort of the spawns by (vector, key): 8-bit digit p is bits
// [8p, 8p + 8) of (vector << 2n) | key.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t wdigit(const WSpawn& r, int p, int n2)
{
    const int b = 8 * p;
    const uint32_t seg = r.meta >> 2;
    if (b < n2) {
        uint32_t d = (uint32_t)(wkey(r) >> b) & 255u;   // key bits at and above 2n are zero
        if (n2 - b < 8) d |= (seg << (n2 - b)) & 255u;
        return d;
    }
    const int sb = b - n2;
    return sb < 32 ? (seg >> sb) & 255u : 0u;
}

__device__ __forceinline__ int64_t spawn_count(const StepParams& P)
{
    return min((int64_t)P.st->spawn_total, P.spawn_cap);
}

__device__ __forceinline__ const WSpawn* pass_src(const WideParams& W, uint32_t plan)
{
    return (plan & 2u) ? W.spawn_alt : W.spawn;
}

// Digit counts of every pass over all spawns (block counts in shared
// memory, then one global add per digit and pass).
__global__ void __launch_bounds__(kWThreads) k_wide_hist(StepParams P, WideParams W)
{
    __shared__ uint32_t h[kWMaxPasses * 256];
    if (cta_error(P.st) || !P.st->sort_fallback) return;
    const int64_t S = spawn_count(P);
    const int n2 = 2 * P.n;
    for (int i = threadIdx.x; i < W.passes * 256; i += blockDim.x) h[i] = 0u;
    __syncthreads();
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < S; i += (int64_t)gridDim.x * blockDim.x) {
        const WSpawn r = wsload(W.spawn, i);
        for (int p = 0; p < W.passes; ++p) atomicAdd(&h[p * 256 + wdigit(r, p, n2)], 1u);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < W.passes * 256; i += blockDim.x)
        if (h[i]) atomicAdd(&W.hist[i], h[i]);
}

// Passes whose digit is the same for every spawn leave the order unchanged:
// skip them.  The others alternate between the two buffers; their digit
// counts become digit starts.  After the bucket sort every pass is skipped
// and the sorted spawns are in spawn_alt.
__global__ void k_wide_plan(StepParams P, WideParams W)
{
    __shared__ uint32_t s_skip;
    if (cta_error(P.st)) return;
    if (!P.st->sort_fallback) {
        for (int p = threadIdx.x; p < W.passes; p += blockDim.x) W.plan[p] = 1u;
        if (threadIdx.x == 0) W.plan[W.passes] = 1u;
        return;
    }
    const uint32_t S = (uint32_t)spawn_count(P);
    uint32_t src = 0;
    for (int p = 0; p < W.passes; ++p) {
        if (threadIdx.x == 0) s_skip = 0u;
        __syncthreads();
        for (int d = threadIdx.x; d < 256; d += blockDim.x)
            if (W.hist[p * 256 + d] == S) s_skip = 1u;
        __syncthreads();
        const bool skip = s_skip != 0u;
        if (threadIdx.x == 0) W.plan[p] = (skip ? 1u : 0u) | (src << 1);
        if (!skip) {
            if (threadIdx.x == 0) {   // counts -> exclusive starts
                uint32_t run = 0;
                for (int d = 0; d < 256; ++d) {
                    const uint32_t c = W.hist[p * 256 + d];
                    W.hist[p * 256 + d] = run;
                    run += c;
                }
            }
            src ^= 1u;
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) W.plan[W.passes] = src;
}

// Per-tile digit counts of one pass.
__global__ void __launch_bounds__(kWThreads) k_wide_tile_hist(StepParams P, WideParams W, int p)
{
    __shared__ uint32_t h[256];
    if (cta_error(P.st)) return;
    const uint32_t plan = W.plan[p];
    if (plan & 1u) return;
    const WSpawn* src = pass_src(W, plan);
    const int64_t S = spawn_count(P);
    const int64_t tiles = (S + kWTile - 1) / kWTile;
    const int n2 = 2 * P.n;
    for (int64_t t = blockIdx.x; t < tiles; t += gridDim.x) {
        h[threadIdx.x] = 0u;
        __syncthreads();
        const int64_t e1 = min(S, (t + 1) * kWTile);
        for (int64_t e = t * kWTile + threadIdx.x; e < e1; e += blockDim.x) atomicAdd(&h[wdigit(src[e], p, n2)], 1u);
        __syncthreads();
        W.tile_hist[t * 256 + threadIdx.x] = h[threadIdx.x];
        __syncthreads();
    }
}

// Per digit (one CTA each): each tile's first output position for that
// digit, the digit's start plus the counts of the tiles before.
__global__ void __launch_bounds__(kWThreads) k_wide_tile_scan(StepParams P, WideParams W, int p)
{
    __shared__ uint32_t wsum[kWThreads / 32];
    if (cta_error(P.st)) return;
    const uint32_t plan = W.plan[p];
    if (plan & 1u) return;
    const int d = blockIdx.x;
    const int64_t S = spawn_count(P);
    const int64_t tiles = (S + kWTile - 1) / kWTile;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t carry = W.hist[p * 256 + d];
    for (int64_t base = 0; base < tiles; base += blockDim.x) {
        const int64_t t = base + threadIdx.x;
        const uint32_t c = t < tiles ? W.tile_hist[t * 256 + d] : 0u;
        uint32_t incl = c;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t v = __shfl_up_sync(kFull, incl, o);
            if (lane >= o) incl += v;
        }
        if (lane == 31) wsum[warp] = incl;
        __syncthreads();
        uint32_t wo = 0, blk = 0;
        for (int q = 0; q < kWThreads / 32; ++q) {
            if (q < warp) wo += wsum[q];
            blk += wsum[q];
        }
        if (t < tiles) W.tile_hist[t * 256 + d] = carry + wo + incl - c;
        carry += blk;
        __syncthreads();
    }
}

// One stable pass: each tile in rounds of kWThreads records; a record's rank
// among equal digits of its round is its warp's offset (prefix over warps in
// thread order) plus its rank among the warp's lanes with that digit.
__global__ void __launch_bounds__(kWThreads) k_wide_scatter(StepParams P, WideParams W, int p)
{
    constexpr int kWarps = kWThreads / 32;
    __shared__ uint32_t s_run[256];
    __shared__ uint32_t s_w[kWarps][256];
    if (cta_error(P.st)) return;
    const uint32_t plan = W.plan[p];
    if (plan & 1u) return;
    const WSpawn* src = pass_src(W, plan);
    WSpawn* dst = (plan & 2u) ? W.spawn : W.spawn_alt;
    const int64_t S = spawn_count(P);
    const int64_t tiles = (S + kWTile - 1) / kWTile;
    const int n2 = 2 * P.n;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (int w = 0; w < kWarps; ++w) s_w[w][tid] = 0u;
    for (int64_t t = blockIdx.x; t < tiles; t += gridDim.x) {
        s_run[tid] = W.tile_hist[t * 256 + tid];
        __syncthreads();
        for (int r = 0; r < kWTile / kWThreads; ++r) {
            const int64_t e = t * kWTile + (int64_t)r * kWThreads + tid;
            const bool valid = e < S;
            WSpawn rec;
            uint32_t d = 256u;
            if (valid) {
                rec = wsload(src, e);
                d = wdigit(rec, p, n2);
            }
            const uint32_t peers = __match_any_sync(kFull, d);
            const uint32_t rank = __popc(peers & lanemask_lt());
            if (valid && lane == __ffs(peers) - 1) s_w[warp][d] = __popc(peers);
            __syncthreads();
            {
                uint32_t run = s_run[tid];
#pragma unroll
                for (int w = 0; w < kWarps; ++w) {
                    const uint32_t c = s_w[w][tid];
                    s_w[w][tid] = run;
                    run += c;
                }
                s_run[tid] = run;
            }
            __syncthreads();
            if (valid) dst[s_w[warp][d] + rank] = rec;
            __syncthreads();
#pragma unroll
            for (int w = 0; w < kWarps; ++w) s_w[w][tid] = 0u;
            __syncthreads();
        }
    }
}

// ---------------------------------------------------------------------------
// Spawn sort by buckets, the default.  The bucket digit holds every vector
// bit and the top bucket_kb key bits, so buckets come in (vector, key) order:
// one counting pass puts each record into its bucket (order inside a bucket
// arbitrary), then the records are cut into windows of whole buckets --
// window k starts at the bucket holding record k kWSortWin -- and every
// window is sorted by (vector, key) in shared memory (a warp for up to
// kWSmallWin records, a CTA for up to kWBigWin).  The order among equal keys
// is irrelevant: a run's records are summed.  When the largest bucket could
// overfill a window the step takes the LSD radix sort instead
// (st->sort_fallback).
// ---------------------------------------------------------------------------
constexpr int kWSortWin = 224;
constexpr int kWSmallWin = 256;
constexpr int kWBigWin = 2048;
constexpr int kWSortRec = 24 + 8 + 8 + 4;   // shared bytes per record: the record, key high, key low, tag
constexpr int kWSmallSmem = (kWThreads / 32) * kWSmallWin * kWSortRec;
constexpr int kWBigSmem = kWBigWin * kWSortRec;

__device__ __forceinline__ uint32_t wbucket(const WSpawn& r, int kb, int n2)
{
    uint32_t d = (r.meta >> 2) << kb;
    if (kb) d |= (uint32_t)(wkey(r) >> (n2 - kb));
    return d;
}

// Bucket sizes of the step's spawns.
__global__ void __launch_bounds__(kWThreads) k_wide_bhist(StepParams P, WideParams W)
{
    DevState* st = P.st;
    if (cta_error(st) || st->sort_fallback) return;
    const int64_t S = spawn_count(P);
    const int kb = P.bucket_kb, n2 = 2 * P.n;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < S; i += (int64_t)gridDim.x * blockDim.x)
        atomicAdd(&P.bucket[wbucket(wsload(W.spawn, i), kb, n2)], 1u);
}

// Per 1024 buckets: their total and largest size, as total | largest << 32.
__global__ void __launch_bounds__(kWThreads) k_wide_bpart(StepParams P)
{
    __shared__ uint32_t ssum[kWThreads / 32], smax[kWThreads / 32];
    DevState* st = P.st;
    if (cta_error(st) || st->sort_fallback) return;
    const int tiles = 1 << (P.bucket_bits - 10);
    for (int t = blockIdx.x; t < tiles; t += gridDim.x) {
        uint32_t c = 0, m = 0;
        for (int b = threadIdx.x; b < 1024; b += blockDim.x) {
            const uint32_t v = P.bucket[t * 1024 + b];
            c += v;
            m = max(m, v);
        }
        c = __reduce_add_sync(kFull, c);
        m = __reduce_max_sync(kFull, m);
        if ((threadIdx.x & 31) == 0) {
            ssum[threadIdx.x >> 5] = c;
            smax[threadIdx.x >> 5] = m;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            uint32_t a = 0, x = 0;
            for (int q = 0; q < kWThreads / 32; ++q) {
                a += ssum[q];
                x = max(x, smax[q]);
            }
            P.bscan_status[t] = (unsigned long long)a | ((unsigned long long)x << 32);
        }
        __syncthreads();
    }
}

// Exclusive prefix of the bucket tiles' totals (one CTA of 1024 threads, at
// most 2^(kBucketBits - 10) tiles); the LSD fallback when the largest bucket
// could overfill a CTA's window.
__global__ void __launch_bounds__(1024) k_wide_btop(StepParams P)
{
    __shared__ uint32_t wsum[32], wmax[32];
    DevState* st = P.st;
    if (cta_error(st) || st->sort_fallback) return;
    const int tiles = 1 << (P.bucket_bits - 10);
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const unsigned long long v = t < tiles ? P.bscan_status[t] : 0ull;
    const uint32_t c = (uint32_t)v, m = (uint32_t)(v >> 32);
    uint32_t incl = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(kFull, incl, o);
        if (lane >= o) incl += y;
    }
    const uint32_t wm = __reduce_max_sync(kFull, m);
    if (lane == 31) wsum[warp] = incl;
    if (lane == 0) wmax[warp] = wm;
    __syncthreads();
    uint32_t off = 0, gm = 0;
    for (int q = 0; q < 32; ++q) {
        if (q < warp) off += wsum[q];
        gm = max(gm, wmax[q]);
    }
    if (t < tiles) P.bscan_status[t] = off + incl - c;
    if (t == 0 && gm > (uint32_t)(kWBigWin - kWSortWin)) st->sort_fallback = 1u;
}

// Bucket starts (exclusive prefix, in place) and the sort windows' starts.
__global__ void __launch_bounds__(1024) k_wide_bapply(StepParams P, WideParams W)
{
    __shared__ uint32_t wsum[32];
    DevState* st = P.st;
    if (cta_error(st) || st->sort_fallback) return;
    const int tiles = 1 << (P.bucket_bits - 10);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int t = blockIdx.x; t < tiles; t += gridDim.x) {
        const int b = t * 1024 + threadIdx.x;
        const uint32_t c = P.bucket[b];
        uint32_t incl = c;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(kFull, incl, o);
            if (lane >= o) incl += y;
        }
        if (lane == 31) wsum[warp] = incl;
        __syncthreads();
        uint32_t off = (uint32_t)P.bscan_status[t];
        for (int q = 0; q < warp; ++q) off += wsum[q];
        const uint32_t start = off + incl - c;
        P.bucket[b] = start;
        for (uint32_t k = (start + kWSortWin - 1) / kWSortWin; k * kWSortWin < start + c; ++k) W.win[k] = start;
        __syncthreads();
    }
}

// Counting pass: spawn -> spawn_alt, each record into its bucket.
__global__ void __launch_bounds__(kWThreads) k_wide_bscatter(StepParams P, WideParams W)
{
    DevState* st = P.st;
    if (cta_error(st) || st->sort_fallback) return;
    const int64_t S = spawn_count(P);
    const int kb = P.bucket_kb, n2 = 2 * P.n;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < S; i += (int64_t)gridDim.x * blockDim.x) {
        const WSpawn r = wsload(W.spawn, i);
        const uint32_t pos = atomicAdd(&P.bucket[wbucket(r, kb, n2)], 1u);
        if ((int64_t)pos < S) W.spawn_alt[pos] = r;
    }
}

// Bitonic sort (N a power of two) by (G >> 12, H, L): G holds the record's
// vector above its 12-bit index in the window, H and L its key's words.
// Threads [t0, N/2) step nthr take the compare-exchanges; sync() orders the
// stages.
template <typename Sync>
__device__ __forceinline__ void wbitonic(uint64_t* H, uint64_t* L, uint32_t* G, int N, int t0, int nthr, Sync sync)
{
    for (int k = 2; k <= N; k <<= 1) {
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int t = t0; t < (N >> 1); t += nthr) {
                const int low = t & (j - 1);
                const int i = ((t - low) << 1) + low;   // bit j of i is clear
                const int l = i + j;
                const bool asc = (i & k) == 0;
                const uint32_t gi = G[i], gl = G[l];
                const uint64_t hi = H[i], hl = H[l], li = L[i], ll = L[l];
                const bool gt = (gi >> 12) != (gl >> 12) ? (gi >> 12) > (gl >> 12)
                                : hi != hl ? hi > hl : li > ll;
                if (gt == asc) {
                    G[i] = gl;
                    G[l] = gi;
                    H[i] = hl;
                    H[l] = hi;
                    L[i] = ll;
                    L[l] = li;
                }
            }
            sync();
        }
    }
}

// Window k's bounds [win[k], win[k + 1]), the last one ending at S.
__device__ __forceinline__ void wwindow(const WideParams& W, int64_t k, int64_t nwin, uint32_t S, uint32_t* lo,
                                        uint32_t* hi)
{
    *lo = W.win[k];
    *hi = k + 1 < nwin ? W.win[k + 1] : S;
}

// Load a window of n records into shared memory (padded to N with keys
// above every record), sort it, write it back in place.
template <typename Sync>
__device__ __forceinline__ void wsort_window(WSpawn* A, uint32_t start, int n, WSpawn* R, uint64_t* H, uint64_t* L,
                                             uint32_t* G, int t0, int nthr, Sync sync)
{
    int N = 2;
    while (N < n) N <<= 1;
    for (int j = t0; j < N; j += nthr) {
        if (j < n) {
            const WSpawn r = wsload(A, start + j);
            R[j] = r;
            H[j] = r.hi;
            L[j] = r.lo;
            G[j] = ((r.meta >> 2) << 12) | (uint32_t)j;
        } else {
            H[j] = ~0ull;
            L[j] = ~0ull;
            G[j] = 0xFFFFF000u | (uint32_t)j;
        }
    }
    sync();
    wbitonic(H, L, G, N, t0, nthr, sync);
    for (int j = t0; j < n; j += nthr) A[start + j] = R[G[j] & 0xFFFu];
    sync();
}

// Windows of up to kWSmallWin records, one warp each; larger windows go to
// the list of k_wide_bsort_big.
__global__ void __launch_bounds__(kWThreads) k_wide_bsort_small(StepParams P, WideParams W)
{
    extern __shared__ __align__(16) uint8_t wsm[];
    DevState* st = P.st;
    if (cta_error(st) || st->sort_fallback) return;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    constexpr int kW = kWThreads / 32;
    WSpawn* R = (WSpawn*)wsm + warp * kWSmallWin;
    uint64_t* H = (uint64_t*)(wsm + kW * kWSmallWin * 24) + warp * kWSmallWin;
    uint64_t* L = (uint64_t*)(wsm + kW * kWSmallWin * 32) + warp * kWSmallWin;
    uint32_t* G = (uint32_t*)(wsm + kW * kWSmallWin * 40) + warp * kWSmallWin;
    const uint32_t S = (uint32_t)spawn_count(P);
    const int64_t nwin = ((int64_t)S + kWSortWin - 1) / kWSortWin;
    for (int64_t k = (int64_t)blockIdx.x * kW + warp; k < nwin; k += (int64_t)gridDim.x * kW) {
        uint32_t start, end;
        wwindow(W, k, nwin, S, &start, &end);
        const int n = (int)(end - start);
        if (n <= 1) continue;
        if (n > kWSmallWin) {
            if (lane == 0) W.big_list[atomicAdd(W.nbig, 1u)] = (uint32_t)k;
            continue;
        }
        wsort_window(W.spawn_alt, start, n, R, H, L, G, lane, 32, [] { __syncwarp(); });
    }
}

// Windows of kWSmallWin + 1 .. kWBigWin records, one CTA each.
__global__ void __launch_bounds__(kWThreads) k_wide_bsort_big(StepParams P, WideParams W)
{
    extern __shared__ __align__(16) uint8_t wsm[];
    WSpawn* R = (WSpawn*)wsm;
    uint64_t* H = (uint64_t*)(wsm + kWBigWin * 24);
    uint64_t* L = (uint64_t*)(wsm + kWBigWin * 32);
    uint32_t* G = (uint32_t*)(wsm + kWBigWin * 40);
    DevState* st = P.st;
    if (cta_error(st) || st->sort_fallback) return;
    const uint32_t S = (uint32_t)spawn_count(P);
    const int64_t nwin = ((int64_t)S + kWSortWin - 1) / kWSortWin;
    const uint32_t nbig = *W.nbig;
    for (uint32_t q = blockIdx.x; q < nbig; q += gridDim.x) {
        uint32_t start, end;
        wwindow(W, (int64_t)W.big_list[q], nwin, S, &start, &end);
        const int n = (int)(end - start);
        if (n > kWBigWin) {   // excluded by the fallback rule
            if (threadIdx.x == 0) set_error(st, DERR_INTERNAL);
            continue;
        }
        wsort_window(W.spawn_alt, start, n, R, H, L, G, threadIdx.x, kWThreads, [] { __syncthreads(); });
    }
}

} // namespace

namespace {

// ---------------------------------------------------------------------------
// Annihilation [End Matter, annihilation step] with the initiator rule
// [End Matter, simulation methodology]: N(t + dt) is the key-ordered union of
// N(t) and the spawn runs, every key's spawns added to its value in N(t); a
// noninitiator's spawn onto a key N(t) does not hold is dropped; zeros go.
// ---------------------------------------------------------------------------

__device__ __forceinline__ const WSpawn* sorted_spawns(const WideParams& W)
{
    return W.plan[W.passes] ? W.spawn_alt : W.spawn;
}

// First index of [lo, hi) of a population slot whose key is >= k.
__device__ __forceinline__ int64_t lower_bound_pop(const ulonglong2* a, int64_t lo, int64_t hi, u128 k)
{
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (wkey(a[mid]) < k) lo = mid + 1; else hi = mid;
    }
    return lo;
}

// Vector boundaries of the sorted spawns: bseg[s] = first spawn of vector >= s.
__global__ void k_wide_spawn_off(StepParams P, WideParams W)
{
    if (cta_error(P.st)) return;
    const WSpawn* sp = sorted_spawns(W);
    const int64_t S = spawn_count(P);
    if (S == 0) {
        for (int s = blockIdx.x * blockDim.x + threadIdx.x; s <= P.nseg; s += gridDim.x * blockDim.x) P.bseg[s] = 0;
        return;
    }
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < S; i += (int64_t)gridDim.x * blockDim.x) {
        const int seg = (int)(sp[i].meta >> 2);
        const int prev = i ? (int)(sp[i - 1].meta >> 2) : -1;
        for (int s = prev + 1; s <= seg; ++s) P.bseg[s] = i;
        if (i == S - 1)
            for (int s = seg + 1; s <= P.nseg; ++s) P.bseg[s] = S;
    }
}

// Where each bucket of the spawn sort starts in N(t): abound[b] = first
// record of b's vector whose key is at least the bucket's smallest key
// (abound[2^bucket_bits] = K), so a spawn's key lies between abound[b] and
// abound[b + 1] of its bucket b.
__global__ void __launch_bounds__(kWThreads) k_wide_abound(StepParams P, WideParams W)
{
    DevState* st = P.st;
    if (cta_error(st) || P.sort_mode == 0) return;
    const int cur = st->cur;
    const WPop A = wpop(P, cur);
    const int64_t* offA = P.segoff[cur];
    const int nb = 1 << P.bucket_bits, kb = P.bucket_kb, n2 = 2 * P.n;
    for (int b = blockIdx.x * blockDim.x + threadIdx.x; b <= nb; b += gridDim.x * blockDim.x) {
        const int seg = b >> kb;
        int64_t p = offA[P.nseg];
        if (b < nb && seg < P.nseg) {
            const u128 lo = kb ? (u128)(uint32_t)(b & ((1 << kb) - 1)) << (n2 - kb) : (u128)0;
            p = lower_bound_pop(A.key, offA[seg], offA[seg + 1], lo);
        }
        W.abound[b] = p;
    }
}

// Runs of equal (vector, key) among the sorted spawns, at their first record.
// A run on a key N(t) holds leaves its spawn sum in delta and, when that
// zeroes the record, counts it in the record's merge tile; a run that brings
// a new key counts it before its position in N(t) and in that tile (one
// atomic per warp when the warp's counts share a tile, as sorted spawns
// mostly do).  The key is looked up in its bucket's stretch of N(t) (its
// whole vector without the bucket digit).
__global__ void __launch_bounds__(kWThreads) k_wide_runs(StepParams P, WideParams W)
{
    DevState* st = P.st;
    if (cta_error(st)) return;
    const WSpawn* sp = sorted_spawns(W);
    const int64_t S = spawn_count(P);
    const int cur = st->cur;
    const WPop A = wpop(P, cur);
    const int64_t* offA = P.segoff[cur];
    const int kb = P.bucket_kb, n2 = 2 * P.n;
    const int lane = threadIdx.x & 31;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31); base < S; base += stride) {
        const int64_t i = base + lane;
        unsigned long long add = 0;   // records zeroed | new keys << 32, for tile `tile`
        int64_t tile = -1;
        if (i < S) {
            const WSpawn r = wsload(sp, i);
            const u128 k = wkey(r);
            const uint32_t seg = r.meta >> 2;
            bool head = true;
            if (i > 0) {
                const WSpawn q = wsload(sp, i - 1);
                head = !((q.meta >> 2) == seg && wkey(q) == k);
            }
            if (!head) {
                W.flag_u[i] = 0;
            } else {
                // the run's end by a galloping search (the spawns after it hold
                // larger (vector, key)), then a sum over that range
                auto same = [&](int64_t j) {
                    const WSpawn q = wsload(sp, j);
                    return (q.meta >> 2) == seg && wkey(q) == k;
                };
                int64_t rend = i + 1, rhi = i + 1, step = 1;   // [i, rend) is the run so far
                while (rhi < S && same(rhi)) {
                    rend = rhi + 1;
                    rhi = min(S, i + 1 + 2 * step - 1);
                    step *= 2;
                }
                while (rend < rhi) {
                    const int64_t mid = (rend + rhi) >> 1;
                    if (same(mid)) rend = mid + 1; else rhi = mid;
                }
                int64_t ire = 0, iim = 0, are = 0, aim = 0;
                for (int64_t j = i; j < rend; ++j) {
                    const WSpawn q = wsload(sp, j);
                    const int64_t v = q.val;
                    const bool to_im = (q.meta >> 1) & 1u;
                    if (to_im) aim += v; else are += v;
                    if (!(q.meta & 1u)) {
                        if (to_im) iim += v; else ire += v;
                    }
                }
                const int64_t hi = offA[seg + 1];
                int64_t lo = offA[seg], top = hi;
                if (P.sort_mode != 0) {
                    const uint32_t bk = wbucket(r, kb, n2);
                    lo = W.abound[bk];
                    top = W.abound[bk + 1];
                }
                const int64_t pos = lower_bound_pop(A.key, lo, top, k);
                const bool matched = pos < hi && wkey(A.key[pos]) == k;
                WRun run;
                run.posA = pos;
                run.re = matched ? are : ire;
                run.im = matched ? aim : iim;
                run.matched = matched ? 1 : 0;
                run.pad = 0;
                W.run[i] = run;
                if (iabs64(run.re) > 2147483647ll || iabs64(run.im) > 2147483647ll) set_error(st, DERR_POP_OVERFLOW);
                const bool fresh = !matched && (ire != 0 || iim != 0);
                if (matched) {
                    W.delta[pos] = make_int2((int32_t)are, (int32_t)aim);   // the one run on this key
                    const int2 a = __ldg(&A.val[pos]);
                    const int64_t vr = (int64_t)a.x + are, vi = (int64_t)a.y + aim;
                    if (iabs64(vr) > 2147483647ll || iabs64(vi) > 2147483647ll) set_error(st, DERR_POP_OVERFLOW);
                    if (vr == 0 && vi == 0) add = 1ull;
                }
                if (fresh) {
                    atomicAdd(&W.newcnt[pos], 1);
                    add = 1ull << 32;
                }
                if (add) tile = pos / kWMTile;
                W.flag_u[i] = fresh ? 1 : 0;
            }
        }
        // the warp's tile counts: one atomic when they share a tile
        const uint32_t act = __ballot_sync(kFull, add != 0);
        if (!act) continue;
        const int64_t t0 = __shfl_sync(kFull, tile, __ffs(act) - 1);
        if (__all_sync(kFull, add == 0 || tile == t0)) {
            const uint32_t kills = __reduce_add_sync(kFull, (uint32_t)add);
            const uint32_t news = __reduce_add_sync(kFull, (uint32_t)(add >> 32));
            if (lane == 0) atomicAdd(&W.mtile[t0], (unsigned long long)kills | ((unsigned long long)news << 32));
        } else if (add) {
            atomicAdd(&W.mtile[tile], add);
        }
    }
}

// Merge tiles over the indices 0 .. K of N(t) (index K carries the new keys
// after the last record).
__device__ __forceinline__ int64_t merge_tiles(int64_t K) { return K / kWMTile + 1; }

// Per merge tile (one CTA): survivors and new keys before it, from the
// counts of the runs kernel (the records of a tile less those its spawns
// zero); clears the counts for the next step; N(t + dt)'s size, with
// POP_CAPACITY when it does not fit.  Each thread sums a contiguous run of
// tiles, one block scan places the runs, the thread writes its tiles' bases.
__device__ __forceinline__ void mtile_counts(const WideParams& W, int64_t t, int64_t K, long long* s, long long* nn)
{
    const unsigned long long m = W.mtile[t];
    const int64_t lo = t * kWMTile, hi = min(K, lo + kWMTile);
    *s = (hi - lo) - (long long)(m & 0xFFFFFFFFull);
    *nn = (long long)(m >> 32);
}

__global__ void __launch_bounds__(1024) k_wide_mtop(StepParams P, WideParams W)
{
    __shared__ long long ws[32], wn[32];
    DevState* st = P.st;
    if (cta_error(st)) return;
    const int64_t K = P.segoff[st->cur][P.nseg];
    const int64_t T = merge_tiles(K);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int64_t per = (T + blockDim.x - 1) / blockDim.x;
    const int64_t t0 = min(T, (int64_t)threadIdx.x * per), t1 = min(T, t0 + per);
    long long s = 0, nn = 0;
#pragma unroll 4
    for (int64_t t = t0; t < t1; ++t) {
        long long a, b;
        mtile_counts(W, t, K, &a, &b);
        s += a;
        nn += b;
    }
    long long is = s, in = nn;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const long long a = __shfl_up_sync(kFull, is, o), b = __shfl_up_sync(kFull, in, o);
        if (lane >= o) {
            is += a;
            in += b;
        }
    }
    if (lane == 31) {
        ws[warp] = is;
        wn[warp] = in;
    }
    __syncthreads();
    long long cs = is - s, cn = in - nn, ts = 0, tn = 0;
    for (int q = 0; q < nw; ++q) {
        if (q < warp) {
            cs += ws[q];
            cn += wn[q];
        }
        ts += ws[q];
        tn += wn[q];
    }
    for (int64_t t = t0; t < t1; ++t) {
        long long a, b;
        mtile_counts(W, t, K, &a, &b);
        W.mtile[t] = 0ull;
        W.mbase[t] = make_longlong2(cs, cn);
        cs += a;
        cn += b;
    }
    if (threadIdx.x == 0) {
        W.mbase[T] = make_longlong2(ts, tn);
        const int64_t total = ts + tn;
        st->next_total = total;
        if (total > st->max_next) st->max_next = total;
        if (total > P.pop_cap) set_error(st, DERR_POP_CAPACITY);
    }
}

// Exclusive prefix sums of the spawns' new-key flags: per-tile sums, their
// prefix (one CTA), the tiles' own prefixes; scan_u[S] is the total.
__global__ void __launch_bounds__(kWThreads) k_wide_scan_part(StepParams P, WideParams W)
{
    __shared__ int64_t red[kWThreads / 32];
    if (cta_error(P.st)) return;
    const int64_t N = spawn_count(P);
    const int64_t tiles = (N + kWScanTile - 1) / kWScanTile;
    for (int64_t t = blockIdx.x; t < tiles; t += gridDim.x) {
        int64_t c = 0;
        const int64_t e1 = min(N, (t + 1) * kWScanTile);
        for (int64_t e = t * kWScanTile + threadIdx.x; e < e1; e += blockDim.x) c += W.flag_u[e];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(kFull, c, o);
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = c;
        __syncthreads();
        if (threadIdx.x == 0) {
            int64_t s = 0;
            for (int q = 0; q < kWThreads / 32; ++q) s += red[q];
            W.part[t] = s;
        }
        __syncthreads();
    }
}

__global__ void __launch_bounds__(kWThreads) k_wide_scan_top(StepParams P, WideParams W)
{
    __shared__ int64_t wsum[kWThreads / 32];
    if (cta_error(P.st)) return;
    const int64_t N = spawn_count(P);
    const int64_t tiles = (N + kWScanTile - 1) / kWScanTile;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int64_t carry = 0;
    for (int64_t base = 0; base < tiles; base += blockDim.x) {
        const int64_t t = base + threadIdx.x;
        const int64_t c = t < tiles ? W.part[t] : 0;
        int64_t incl = c;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int64_t v = __shfl_up_sync(kFull, incl, o);
            if (lane >= o) incl += v;
        }
        if (lane == 31) wsum[warp] = incl;
        __syncthreads();
        int64_t wo = 0, blk = 0;
        for (int q = 0; q < kWThreads / 32; ++q) {
            if (q < warp) wo += wsum[q];
            blk += wsum[q];
        }
        if (t < tiles) W.part[t] = carry + wo + incl - c;
        carry += blk;
        __syncthreads();
    }
    if (threadIdx.x == 0) W.scan_u[N] = carry;
}

__global__ void __launch_bounds__(kWThreads) k_wide_scan_apply(StepParams P, WideParams W)
{
    constexpr int kPer = kWScanTile / kWThreads;
    __shared__ int64_t wsum[kWThreads / 32];
    if (cta_error(P.st)) return;
    const int64_t N = spawn_count(P);
    const int64_t tiles = (N + kWScanTile - 1) / kWScanTile;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int64_t t = blockIdx.x; t < tiles; t += gridDim.x) {
        // each thread a run of kPer consecutive flags
        const int64_t e0 = t * kWScanTile + (int64_t)threadIdx.x * kPer;
        int64_t v[kPer];
        int64_t c = 0;
#pragma unroll
        for (int k = 0; k < kPer; ++k) {
            v[k] = e0 + k < N ? W.flag_u[e0 + k] : 0;
            c += v[k];
        }
        int64_t incl = c;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int64_t x = __shfl_up_sync(kFull, incl, o);
            if (lane >= o) incl += x;
        }
        if (lane == 31) wsum[warp] = incl;
        __syncthreads();
        int64_t run = W.part[t];
        for (int q = 0; q < warp; ++q) run += wsum[q];
        run += incl - c;
#pragma unroll
        for (int k = 0; k < kPer; ++k) {
            if (e0 + k < N) W.scan_u[e0 + k] = run;
            run += v[k];
        }
        __syncthreads();
    }
}

} // namespace

namespace {

// Per-vector observables of N(t + dt) as the merge writes it: records,
// N_tot = sum |re| + |im|, and the diagonal sums, accumulated per thread
// while its vector stays the same.
struct ObsAcc {
    int seg = -1;
    unsigned long long c = 0;
    long long ntot = 0, dre = 0, dim = 0;

    __device__ __forceinline__ void add(const ulonglong2& key, int2 v, int n)
    {
        ++c;
        ntot += (v.x < 0 ? -(long long)v.x : v.x) + (v.y < 0 ? -(long long)v.y : v.y);
        const u128 k = wkey(key);
        if ((uint64_t)(k >> n) == ((uint64_t)k & ((1ull << n) - 1ull))) {
            dre += v.x;
            dim += v.y;
        }
    }

    __device__ __forceinline__ void flush(SegStats* out)
    {
        if (seg >= 0 && c) {
            atomicAdd(&out[seg].count, c);
            atomicAdd((unsigned long long*)&out[seg].ntot, (unsigned long long)ntot);
            atomicAdd((unsigned long long*)&out[seg].dre, (unsigned long long)dre);
            atomicAdd((unsigned long long*)&out[seg].dim, (unsigned long long)dim);
        }
        c = 0;
        ntot = dre = dim = 0;
    }

    // Last flush of a kernel (all lanes of the warp): one lane's atomics when
    // the warp shares its vector.
    __device__ __forceinline__ void flush_warp(SegStats* out)
    {
        const int s0 = __shfl_sync(kFull, seg, 0);
        if (__all_sync(kFull, seg == s0)) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                c += __shfl_xor_sync(kFull, c, o);
                ntot += __shfl_xor_sync(kFull, ntot, o);
                dre += __shfl_xor_sync(kFull, dre, o);
                dim += __shfl_xor_sync(kFull, dim, o);
            }
            if ((threadIdx.x & 31) != 0) c = 0;
        }
        flush(out);
    }
};

// N(t) into N(t + dt), one pass over every merge tile [End Matter,
// annihilation step]: each record's value plus the spawn sum of its run
// (delta); survivors (nonzero) go to their place in the key-ordered union,
// after the survivors and new keys before them and the new keys just before
// them.  The places come from the tile's bases and a prefix over the tile,
// kWMBatch rounds of kWThreads indices at a time (the batch's loads issued
// together, one barrier per batch).  Where new keys go just before a record,
// and at the first record of every vector, the survivors before it are left
// in scan_a for the new keys' scatter and the vector offsets.  delta and
// newcnt are cleared where set.  Each CTA takes a contiguous range of tiles.
constexpr int kWMBatch = 4;

__global__ void __launch_bounds__(kWThreads, 3) k_wide_merge_a(StepParams P, WideParams W)
{
    constexpr int kWarps = kWThreads / 32;
    constexpr int kSpan = kWMBatch * kWThreads;
    __shared__ unsigned long long s_w[2][kWMBatch][kWarps];
    DevState* st = P.st;
    if (cta_error(st)) return;
    const int cur = st->cur;
    const WPop A = wpop(P, cur);
    const WPop out = wpop(P, (cur + 1) % 3);
    const int64_t* offA = P.segoff[cur];
    const int64_t K = offA[P.nseg];
    const int64_t T = merge_tiles(K);
    const int64_t per = (T + gridDim.x - 1) / gridDim.x;
    const int64_t tb = (int64_t)blockIdx.x * per, te = min(T, tb + per);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    ObsAcc acc;
    int n = 0;
    int64_t seg_lo = 0, seg_hi = 0;
    int par = 0;
    for (int64_t t = tb; t < te; ++t) {
        const longlong2 base = W.mbase[t];
        unsigned long long carry = 0;   // survivors | new keys << 32 of the tile's earlier indices
        for (int r = 0; r < kWMTile / kSpan; ++r) {
            const int64_t r0 = t * kWMTile + (int64_t)r * kSpan;
            if (r0 > K) break;   // same for the whole CTA
            int nc[kWMBatch];
            int2 v[kWMBatch];
            ulonglong2 key[kWMBatch];
            unsigned long long x[kWMBatch], incl[kWMBatch];
#pragma unroll
            for (int b = 0; b < kWMBatch; ++b) {
                const int64_t i = r0 + b * kWThreads + tid;
                nc[b] = i <= K ? W.newcnt[i] : 0;
                int2 d = make_int2(0, 0), a = make_int2(0, 0);
                key[b] = make_ulonglong2(0ull, 0ull);
                if (i < K) {
                    d = W.delta[i];
                    a = __ldg(&A.val[i]);
                    key[b] = __ldg(&A.key[i]);
                }
                v[b] = make_int2(a.x + d.x, a.y + d.y);   // range checked by the runs kernel
                if (d.x | d.y) W.delta[i] = make_int2(0, 0);
                if (nc[b]) W.newcnt[i] = 0;
                x[b] = ((v[b].x | v[b].y) != 0 ? 1ull : 0ull) | ((unsigned long long)(uint32_t)nc[b] << 32);
                incl[b] = x[b];
            }
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
#pragma unroll
                for (int b = 0; b < kWMBatch; ++b) {
                    const unsigned long long y = __shfl_up_sync(kFull, incl[b], o);
                    if (lane >= o) incl[b] += y;
                }
            }
            if (lane == 31) {
#pragma unroll
                for (int b = 0; b < kWMBatch; ++b) s_w[par][b][warp] = incl[b];
            }
            __syncthreads();
#pragma unroll
            for (int b = 0; b < kWMBatch; ++b) {
                unsigned long long wo = 0, blk = 0;
#pragma unroll
                for (int q = 0; q < kWarps; ++q) {
                    const unsigned long long u = s_w[par][b][q];
                    if (q < warp) wo += u;
                    blk += u;
                }
                const unsigned long long ex = carry + wo + incl[b] - x[b];
                carry += blk;
                const int64_t i = r0 + b * kWThreads + tid;
                if (i > K) continue;
                const int64_t surv = base.x + (int64_t)(ex & 0xFFFFFFFFull);
                const int64_t newb = base.y + (int64_t)(ex >> 32);
                bool start = i == K;
                if (i < K) {
                    if (acc.seg < 0 || i >= seg_hi) {
                        acc.flush(P.segacc);
                        acc.seg = seg_of(offA, P.nseg, i);
                        seg_lo = offA[acc.seg];
                        seg_hi = offA[acc.seg + 1];
                        n = P.seginfo[acc.seg].n;
                    }
                    start = i == seg_lo;
                }
                if (nc[b] > 0 || start) W.scan_a[i] = surv;
                if (x[b] & 1ull) {
                    const int64_t o = surv + newb + nc[b];
                    if (o < P.pop_cap) {
                        out.key[o] = key[b];
                        out.val[o] = v[b];
                        acc.add(key[b], v[b], n);
                    } else {
                        set_error(st, DERR_POP_CAPACITY);
                    }
                }
            }
            par ^= 1;
        }
        // self-check: the tile's survivors and new keys as the runs counted them
        if (tid == 0) {
            const longlong2 nx = W.mbase[t + 1];
            if (nx.x - base.x != (long long)(carry & 0xFFFFFFFFull) || nx.y - base.y != (long long)(carry >> 32))
                set_error(st, DERR_INTERNAL);
        }
    }
    acc.flush_warp(P.segacc);
}

// The new keys of N(t + dt): run j after the new keys before it and the
// survivors of N(t) before its position there.  Each CTA a contiguous range.
__global__ void __launch_bounds__(kWThreads) k_wide_scatter_u(StepParams P, WideParams W)
{
    DevState* st = P.st;
    if (cta_error(st)) return;
    const int cur = st->cur;
    const WSpawn* sp = sorted_spawns(W);
    const WPop out = wpop(P, (cur + 1) % 3);
    const int64_t S = spawn_count(P);
    const int64_t per = (S + gridDim.x - 1) / gridDim.x;
    const int64_t b0 = (int64_t)blockIdx.x * per, b1 = min(S, b0 + per);
    ObsAcc acc;
    int n = 0;
    for (int64_t i = b0 + threadIdx.x; i < b1; i += blockDim.x) {
        if (!W.flag_u[i]) continue;
        const WRun run = W.run[i];
        const int64_t o = W.scan_u[i] + W.scan_a[run.posA];
        const WSpawn r = wsload(sp, i);
        const int seg = (int)(r.meta >> 2);
        if (seg != acc.seg) {
            acc.flush(P.segacc);
            acc.seg = seg;
            n = P.seginfo[seg].n;
        }
        const ulonglong2 key = make_ulonglong2(r.lo, r.hi);
        const int2 v = make_int2((int32_t)run.re, (int32_t)run.im);
        if (o < P.pop_cap) {
            out.key[o] = key;
            out.val[o] = v;
            acc.add(key, v, n);
        } else {
            set_error(st, DERR_POP_CAPACITY);
        }
    }
    acc.flush_warp(P.segacc);
}

// Vector offsets of N(t + dt): survivors of N(t) before vector s plus the new
// keys before it.
__global__ void k_wide_outoff(StepParams P, WideParams W)
{
    DevState* st = P.st;
    if (cta_error(st)) return;
    const int cur = st->cur, nxt = (cur + 1) % 3;
    const int64_t* offA = P.segoff[cur];
    int64_t* off = P.segoff[nxt];
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s <= P.nseg; s += gridDim.x * blockDim.x)
        off[s] = W.scan_a[offA[s]] + W.scan_u[P.bseg[s]];
}

// Per-vector K, N_tot and N^diag of a slot: each CTA a contiguous range, a
// thread accumulating while its vector stays the same.
__global__ void __launch_bounds__(kWThreads) k_wide_obs(StepParams P, int slot_rel, SegStats* __restrict__ out)
{
    const DevState* st = P.st;
    if (read_error(st)) return;
    const int slot = (st->cur + slot_rel) % 3;
    const WPop pop = wpop(P, slot);
    const int64_t* off = P.segoff[slot];
    const int64_t K = off[P.nseg];
    const int64_t per = (K + gridDim.x - 1) / gridDim.x;
    const int64_t b0 = (int64_t)blockIdx.x * per, b1 = min(K, b0 + per);
    int cs = -1, n = 0;
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
            c = 0;
            ntot = dre = dim = 0;
        }
        const WRec r = wload(pop, i);
        ++c;
        ntot += (r.re < 0 ? -(long long)r.re : r.re) + (r.im < 0 ? -(long long)r.im : r.im);
        const u128 k = wkey(r);
        if ((uint64_t)(k >> n) == ((uint64_t)k & ((1ull << n) - 1ull))) {
            dre += r.re;
            dim += r.im;
        }
    }
    flush();
}

// History of the step, counters, rotation (single CTA).
__global__ void k_wide_finalize(StepParams P)
{
    DevState* st = P.st;
    if (cta_error(st)) return;
    const int cur = st->cur, nxt = (cur + 1) % 3;
    const int ci = st->call_index;
    long long walkers = 0;
    for (int s = threadIdx.x; s < P.nseg; s += blockDim.x) {
        const SegStats h = P.segacc[s];
        if (ci < P.history_cap) {
            P.history[(int64_t)ci * P.nseg + s] = h;
            long long* zh = P.zhist + ((int64_t)ci * P.nseg + s) * P.n;
            for (int q = 0; q < P.n; ++q) zh[q] = 0ll;   // <Z_q> sums: not reduced on this path
        }
        walkers += h.ntot;
    }
    __shared__ long long wsum;
    if (threadIdx.x == 0) wsum = 0;
    __syncthreads();
    atomicAdd((unsigned long long*)&wsum, (unsigned long long)walkers);
    __syncthreads();
    if (threadIdx.x == 0) {
        const StepInfo inf = P.info[ci];
        const int64_t next = P.segoff[nxt][P.nseg];
        st->acc_steps += 1;
        st->acc_walkers += wsum;
        st->acc_kcur += st->count[cur];
        st->acc_kprev += inf.ab2 ? st->count[(cur + 2) % 3] : 0;
        st->acc_spawn += st->spawn_total;
        st->acc_knext += next;
        st->acc_heavy += st->heavy_total;
        st->acc_cand += st->cand_total;
        if (st->sort_fallback) st->acc_sort_lsd += 1; else st->acc_sort_bucket += 1;
        if (st->cand_total > st->max_cand) st->max_cand = st->cand_total;
        if (st->spawn_total > st->max_spawn) st->max_spawn = st->spawn_total;
        if (st->heavy_total > st->max_heavy) st->max_heavy = st->heavy_total;
        st->count[nxt] = next;
        st->cur = nxt;
        st->step += 1;
        st->call_index += 1;
    }
}

// The observables of N(t + dt) go into segacc: the slot after the current one.
__global__ void k_wide_zero_hist(WideParams W)
{
    for (int i = threadIdx.x; i < kWMaxPasses * 256; i += blockDim.x) W.hist[i] = 0u;
    if (threadIdx.x == 0) *W.nbig = 0u;
}

int g_wide_grid = 0;

int wide_grid()
{
    if (!g_wide_grid) {
        int dev = 0, sms = 1;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        g_wide_grid = sms * 8;
    }
    return g_wide_grid;
}

} // namespace

void configure_wide_kernels()
{
    (void)wide_grid();
    cudaFuncSetAttribute(k_wide_bsort_small, cudaFuncAttributeMaxDynamicSharedMemorySize, kWSmallSmem);
    cudaFuncSetAttribute(k_wide_bsort_big, cudaFuncAttributeMaxDynamicSharedMemorySize, kWBigSmem);
}

// The kernels of one step, in order, on one stream (captured into a graph by
// the host).
const char* const kWideGroupNames[kNumWideGroups] = {
    "w_prologue", "w_spawn", "w_spawn_heavy", "w_sort_hist_plan", "w_sort_passes",
    "w_merge_runs", "w_merge_scans", "w_merge_scatter", "w_finalize"};

void launch_wide_step(const StepParams& P, const WideParams& W, cudaStream_t s, cudaEvent_t* ev)
{
    const int g = wide_grid();
    auto mark = [&](int i) {
        if (ev) cudaEventRecord(ev[i], s);
    };
    mark(0);
    k_wide_prologue<<<1, kWThreads, 0, s>>>(P);
    k_wide_zero_hist<<<1, kWThreads, 0, s>>>(W);
    k_wide_abound<<<g, kWThreads, 0, s>>>(P, W);
    mark(1);
    k_wide_spawn<<<g, kWThreads, 0, s>>>(P, W, 0);
    k_wide_spawn<<<g, kWThreads, 0, s>>>(P, W, 1);
    k_wide_choose<<<g, kWThreads, 0, s>>>(P, W);
    mark(2);
    k_wide_heavy<<<g, kWThreads, 0, s>>>(P, W);
    mark(3);
    k_wide_bhist<<<g, kWThreads, 0, s>>>(P, W);
    k_wide_bpart<<<g, kWThreads, 0, s>>>(P);
    k_wide_btop<<<1, 1024, 0, s>>>(P);
    k_wide_bapply<<<g, 1024, 0, s>>>(P, W);
    k_wide_bscatter<<<g, kWThreads, 0, s>>>(P, W);
    k_wide_bsort_small<<<g, kWThreads, kWSmallSmem, s>>>(P, W);
    k_wide_bsort_big<<<g, kWThreads, kWBigSmem, s>>>(P, W);
    k_wide_hist<<<g, kWThreads, 0, s>>>(P, W);
    k_wide_plan<<<1, kWThreads, 0, s>>>(P, W);
    mark(4);
    for (int p = 0; p < W.passes; ++p) {
        k_wide_tile_hist<<<g, kWThreads, 0, s>>>(P, W, p);
        k_wide_tile_scan<<<256, kWThreads, 0, s>>>(P, W, p);
        k_wide_scatter<<<g, kWThreads, 0, s>>>(P, W, p);
    }
    mark(5);
    k_wide_spawn_off<<<g, kWThreads, 0, s>>>(P, W);
    k_wide_runs<<<g, kWThreads, 0, s>>>(P, W);
    k_wide_mtop<<<1, 1024, 0, s>>>(P, W);
    mark(6);
    k_wide_scan_part<<<g, kWThreads, 0, s>>>(P, W);
    k_wide_scan_top<<<1, kWThreads, 0, s>>>(P, W);
    k_wide_scan_apply<<<g, kWThreads, 0, s>>>(P, W);
    mark(7);
    k_wide_merge_a<<<g, kWThreads, 0, s>>>(P, W);
    k_wide_scatter_u<<<g, kWThreads, 0, s>>>(P, W);
    k_wide_outoff<<<1, kWThreads, 0, s>>>(P, W);
    mark(8);
    k_wide_finalize<<<1, kWThreads, 0, s>>>(P);
    mark(9);
}

int wide_step_launch_count(const StepParams& P, const WideParams& W)
{
    (void)P;
    return 16 + 3 * W.passes + 3 + 3 + 3 + 1;
}

namespace {

// N(0) = N^diag rho(0), stochastic rounding per component [walker averaging,
// Eq. (3); reading R4]: the draw of element (x, y) is keyed by the 128-bit
// key, bits 0-63 in the first two counter words, 64-95 in the fourth and
// 96-119 in the top 24 bits of the third.
__global__ void k_wide_init_values(StepParams P, const uint64_t* __restrict__ xs, const uint64_t* __restrict__ ys,
                                   const double* __restrict__ re, const double* __restrict__ im, int64_t nnz,
                                   int64_t* __restrict__ vals)
{
    const int64_t total = nnz * P.nseg;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const int s = (int)(i / nnz);
        const int64_t e = i - (int64_t)s * nnz;
        const SegInfo si = P.seginfo[s];
        const InstInfo in = P.inst[si.inst];
        const uint4 kk = philox10(make_uint4(0u, 0u, (uint32_t)si.vec, kTagInit),
                                  make_uint2((uint32_t)in.seed, (uint32_t)(in.seed >> 32)));
        const uint2 kd = make_uint2(kk.x, kk.y);
        const u128 key = ((u128)xs[e] << si.n) | (u128)ys[e];
        for (int comp = 0; comp < 2; ++comp) {
            const double v = __dmul_rn((double)in.n_diag, comp ? im[e] : re[e]);
            const double fl = floor(v);
            const double fr = __dsub_rn(v, fl);
            const uint4 w = philox10(make_uint4((uint32_t)key, (uint32_t)(key >> 32),
                                                ((uint32_t)comp << 1) | (kKindInit << 2) |
                                                    ((uint32_t)(key >> 96) << 8),
                                                (uint32_t)(key >> 64)),
                                     kd);
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

// Nonzero values per vector into slot cur, in input (= key) order (one CTA).
__global__ void k_wide_init_compact(StepParams P, const uint64_t* __restrict__ xs, const uint64_t* __restrict__ ys,
                                    int64_t nnz, const int64_t* __restrict__ vals)
{
    __shared__ int s_cnt[kWThreads];
    DevState* st = P.st;
    const int slot = st->cur;
    const WPop dst = wpop(P, slot);
    int64_t* off = P.segoff[slot];
    int64_t pos = 0;
    const int tid = threadIdx.x;
    for (int s = 0; s < P.nseg; ++s) {
        if (tid == 0) off[s] = pos;
        const int n = P.seginfo[s].n;
        for (int64_t base = 0; base < nnz; base += kWThreads) {
            const int64_t e = base + tid;
            const int64_t i = (int64_t)s * nnz + e;
            const bool keep = e < nnz && (vals[2 * i] != 0 || vals[2 * i + 1] != 0);
            s_cnt[tid] = keep ? 1 : 0;
            __syncthreads();
            for (int o = 1; o < kWThreads; o <<= 1) {
                const int v = tid >= o ? s_cnt[tid - o] : 0;
                __syncthreads();
                s_cnt[tid] += v;
                __syncthreads();
            }
            const int excl = s_cnt[tid] - (keep ? 1 : 0);
            const int blk = s_cnt[kWThreads - 1];
            if (keep && pos + excl < P.pop_cap)
                wstore(dst, pos + excl, ((u128)xs[e] << n) | (u128)ys[e], (int32_t)vals[2 * i],
                       (int32_t)vals[2 * i + 1]);
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

// Values of query states |qx><qy| in one vector of N(t) (0 when absent).
__global__ void k_wide_lookup(StepParams P, int seg, const uint64_t* __restrict__ qx, const uint64_t* __restrict__ qy,
                              int nq, int64_t* __restrict__ out)
{
    const int cur = P.st->cur;
    const WPop A = wpop(P, cur);
    const int64_t lo = P.segoff[cur][seg], hi = P.segoff[cur][seg + 1];
    const int n = P.seginfo[seg].n;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nq; i += gridDim.x * blockDim.x) {
        const u128 k = ((u128)qx[i] << n) | (u128)qy[i];
        const int64_t p = lower_bound_pop(A.key, lo, hi, k);
        const bool hit = p < hi && wkey(A.key[p]) == k;
        const int2 v = hit ? A.val[p] : make_int2(0, 0);
        out[2 * i] = v.x;
        out[2 * i + 1] = v.y;
    }
}

__global__ void k_wide_export(StepParams P, int slot, int64_t first, int64_t count, uint64_t* __restrict__ x,
                              uint64_t* __restrict__ y, int32_t* __restrict__ re, int32_t* __restrict__ im)
{
    const WPop A = wpop(P, slot);
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x) {
        const WRec r = wload(A, first + i);
        const int seg = seg_of(P.segoff[slot], P.nseg, first + i);
        const int n = P.seginfo[seg].n;
        const u128 k = wkey(r);
        x[i] = (uint64_t)(k >> n);
        y[i] = (uint64_t)k & ((1ull << n) - 1ull);
        re[i] = r.re;
        im[i] = r.im;
    }
}

} // namespace

void launch_wide_init(const StepParams& P, const uint64_t* xs, const uint64_t* ys, const double* re,
                      const double* im, int64_t nnz, int64_t* vals, cudaStream_t s)
{
    if (nnz > 0) k_wide_init_values<<<wide_grid(), kWThreads, 0, s>>>(P, xs, ys, re, im, nnz, vals);
    k_wide_init_compact<<<1, kWThreads, 0, s>>>(P, xs, ys, nnz, vals);
}

void launch_wide_obs(const StepParams& P, int which, SegStats* out, cudaStream_t s)
{
    // which 0: N(t) (slot cur), 1: N(t - dt) (slot cur + 2)
    k_wide_obs<<<wide_grid(), kWThreads, 0, s>>>(P, which ? 2 : 0, out);
}

void launch_wide_lookup(const StepParams& P, int seg, const uint64_t* qx, const uint64_t* qy, int nq, int64_t* out,
                        cudaStream_t s)
{
    if (nq > 0) k_wide_lookup<<<(nq + kWThreads - 1) / kWThreads, kWThreads, 0, s>>>(P, seg, qx, qy, nq, out);
}

void launch_wide_export(const StepParams& P, int slot, int64_t first, int64_t count, uint64_t* x, uint64_t* y,
                        int32_t* re, int32_t* im, cudaStream_t s)
{
    if (count > 0) k_wide_export<<<wide_grid(), kWThreads, 0, s>>>(P, slot, first, count, x, y, re, im);
}

} // namespace qmc

namespace qmc {

namespace {

// Records |x><y| of the caller into a population slot; bad is set for a state
// beyond n qubits, a zero or INT32_MIN value, or keys not ascending inside a
// vector.
__global__ void k_wide_pack(const uint64_t* __restrict__ xs, const uint64_t* __restrict__ ys,
                            const int32_t* __restrict__ re, const int32_t* __restrict__ im,
                            const int64_t* __restrict__ off, int nseg, const SegInfo* __restrict__ seginfo,
                            uint8_t* __restrict__ dst_base, int64_t cap, int* bad)
{
    const int64_t K = off[nseg];
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < K; i += (int64_t)gridDim.x * blockDim.x) {
        const int s = seg_of(off, nseg, i);
        const int n = seginfo[s].n;
        const uint64_t lim = (1ull << n) - 1ull;
        const int32_t a = re[i], b = im[i];
        bool ok = (xs[i] & ~lim) == 0 && (ys[i] & ~lim) == 0 && (a != 0 || b != 0) && a != INT32_MIN && b != INT32_MIN;
        const u128 k = ((u128)xs[i] << n) | (u128)ys[i];
        if (ok && i > off[s]) {
            const u128 kp = ((u128)xs[i - 1] << n) | (u128)ys[i - 1];
            if (kp >= k) ok = false;
        }
        if (!ok) atomicExch(bad, 1);
        const WPop dst{(ulonglong2*)dst_base, (int2*)(dst_base + 16 * cap)};
        wstore(dst, i, k, a, b);
    }
}

} // namespace

void launch_wide_pack(const uint64_t* xs, const uint64_t* ys, const int32_t* re, const int32_t* im,
                      const int64_t* off, int nseg, const SegInfo* seginfo, uint8_t* dst, int64_t cap, int* bad,
                      cudaStream_t s)
{
    k_wide_pack<<<wide_grid(), kWThreads, 0, s>>>(xs, ys, re, im, off, nseg, seginfo, dst, cap, bad);
}

} // namespace qmc
