// The step for 33..60 qubits, where a key (x << n) | y needs 128 bits
// (arXiv:2502.18929: the method of the 64-bit step, same random stream).
//
//   k_wide_prologue     per-step Philox keys, counter resets
//   k_wide_spawn        spawning [End Matter, spawn step] of parents with few
//                       walkers, one thread per parent, a warp's spawns
//                       appended together; heavy parents become work items
//   k_wide_heavy        one warp per chunk of a heavy parent's walkers
//   k_wide_hist         digit counts of every 8-bit radix pass of (vector, key)
//   k_wide_plan         passes to skip (a digit shared by every record) and
//                       the ping-pong buffer of each pass
//   k_wide_tile_hist /
//   k_wide_tile_scan /
//   k_wide_scatter      one stable LSD pass: per-tile counts, their prefix
//                       over tiles per digit, scatter with warp-match ranks
//   k_wide_spawn_off    vector boundaries of the sorted spawns
//   k_wide_runs         runs of equal keys: summed spawns under the initiator
//                       rule, the key's position in N(t)
//   k_wide_match        each record of N(t) with the spawns on its key
//   k_wide_scan_*       exclusive prefix sums of the survivors
//   k_wide_scatter_*    N(t + dt) = the survivors in key order [End Matter,
//                       annihilation step], with the per-vector observables
//   k_wide_finalize     vector offsets of N(t + dt), history, rotate the slots
//
// Integer-only, like the 64-bit step: results are bit-identical to the
// oracle whatever the launch shape.
#include <cuda_runtime.h>
#include <stdint.h>

#include "column_eval.h"
#include "device_common.h"
#include "kernels.h"

namespace qmc {

namespace {

constexpr int kWThreads = 256;

__device__ __forceinline__ u128 wkey(uint64_t lo, uint64_t hi) { return ((u128)hi << 64) | (u128)lo; }
__device__ __forceinline__ u128 wkey(const WRec& r) { return wkey(r.lo, r.hi); }
__device__ __forceinline__ u128 wkey(const WSpawn& r) { return wkey(r.lo, r.hi); }

__device__ __forceinline__ WRec wload(const WRec* p, int64_t i)
{
    WRec r;
    r.lo = __ldg(&p[i].lo);
    r.hi = __ldg(&p[i].hi);
    const int2 v = __ldg((const int2*)&p[i].re);
    r.re = v.x;
    r.im = v.y;
    return r;
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

// One parent as its walkers see it.
struct WParent {
    uint64_t x, y;
    u128 key;
    int32_t re, im;
    uint32_t rank;
    int seg, phase;
    int64_t Pw, sre, sim;
    int noninit;
    uint2 kd;
};

// Parent i of a slot: its state, column weight and initiator status.  Returns
// false (after raising the error) when its spawn probability reaches 1.
__device__ bool load_parent(const StepParams& P, const StepInfo& inf, const WRec* pop, const int64_t* off, int64_t i,
                            int phase, WParent* q, WProg* pr)
{
    const WRec r = wload(pop, i);
    const int seg = seg_of(off, P.nseg, i);
    const SegInfo si = P.seginfo[seg];
    const int n = si.n;
    q->key = wkey(r);
    q->x = (uint64_t)(q->key >> n);
    q->y = (uint64_t)q->key & ((1ull << n) - 1ull);
    q->re = r.re;
    q->im = r.im;
    q->rank = (uint32_t)(i - off[seg]);
    q->seg = seg;
    q->phase = phase;
    q->kd = P.kd[seg];
    *pr = wprog_at(prog_of(P, inf, si.inst, phase));
    q->Pw = column_weight(*pr, q->x, q->y, &q->sre, &q->sim);
    const int64_t m = iabs64(r.re) + iabs64(r.im);
    const int64_t init_min = P.inst[si.inst].init_min;
    q->noninit = (init_min > 0 && m < init_min) ? 1 : 0;
    if (q->Pw >= (1ll << 52)) {
        set_error(P.st, DERR_DT_TOO_LARGE);
        return false;
    }
    return true;
}

// Walker w of a parent (real walkers first) with its 32-bit word W: the
// prefilter W <= (P - 1) >> 20, then the full draw T = W << 20 | L [reading
// R3]; if T < P the spawn record of the destination whose cumulative-weight
// interval holds T, with the paper's sign rule [End Matter, spawn step].
__device__ __forceinline__ bool wide_walker(const WProg& pr, const WParent& q, int64_t w, uint32_t W, WSpawn* out)
{
    if ((int64_t)W > ((q.Pw - 1) >> 20)) return false;
    const int64_t are = iabs64(q.re);
    const int comp = w < are ? 0 : 1;
    const uint32_t j = (uint32_t)(comp ? w - are : w);
    const int64_t T = walker_T(W, q.rank, j, comp, q.phase, q.kd);
    if (T >= q.Pw) return false;
    u128 mask;
    int chan;
    int64_t v;
    if (!choose_destination(pr, q.x, q.y, q.sre, q.sim, T, &mask, &chan, &v)) return false;
    const int sg = comp == 0 ? (q.re > 0 ? 1 : -1) : (q.im > 0 ? 1 : -1);
    const int s = (q.phase ? -1 : 1) * sg * (v > 0 ? 1 : -1);
    int target, val;
    if (chan == 0) { target = comp; val = s; }
    else if (comp == 0) { target = 1; val = s; }
    else { target = 0; val = -s; }
    const u128 dest = q.key ^ mask;
    out->lo = (uint64_t)dest;
    out->hi = (uint64_t)(dest >> 64);
    out->meta = ((uint32_t)q.seg << 2) | ((uint32_t)target << 1) | (uint32_t)q.noninit;
    out->val = val;
    return true;
}

// The 32-bit word of walker w (w = 0, 1: the rank group's call of level w;
// w >= 2: the parent's call (w - 2) / 4).
__device__ __forceinline__ uint32_t walker_word(const WParent& q, int64_t w)
{
    if (w <= 1) return word_of(group_words(q.rank >> 2, (uint32_t)w, q.phase, q.kd), (int)(q.rank & 3u));
    return word_of(extra_words(q.rank, (uint32_t)((w - 2) >> 2), q.phase, q.kd), (int)((w - 2) & 3));
}

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
    if (threadIdx.x == 0) {
        st->spawn_total = 0;
        st->cand_total = 0;
        st->heavy_total = 0;
        st->next_total = 0;
        st->merge_tiles = 0;
    }
}

// ---------------------------------------------------------------------------
// Spawning of light parents: one thread per parent, the warp's lanes stepping
// through their walkers together so that each round's spawns take one atomic.
// A parent with more than kWLight walkers becomes heavy work items of
// kWChunk walkers each.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kWThreads) k_wide_spawn(StepParams P, WideParams W, int phase)
{
    DevState* st = P.st;
    if (cta_error(st)) return;
    const StepInfo inf = P.info[st->call_index];
    if (phase == 1 && !inf.ab2) return;
    const int slot = phase ? (st->cur + 2) % 3 : st->cur;
    const WRec* pop = (const WRec*)P.pop[slot];
    const int64_t* off = P.segoff[slot];
    const int64_t K = off[P.nseg];
    const int lane = threadIdx.x & 31;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31); base < K; base += stride) {
        const int64_t i = base + lane;
        WParent q;
        WProg pr;
        int64_t m = 0;
        if (i < K) {
            if (load_parent(P, inf, pop, off, i, phase, &q, &pr)) {
                m = iabs64(q.re) + iabs64(q.im);
                if (m > kWLight) {
                    const int64_t nb = (m - 2 + 3) / 4;   // extra calls (m > kWLight >= 2)
                    const int64_t chunks = (nb + kWChunk - 1) / kWChunk;
                    const int64_t at =
                        (int64_t)atomicAdd((unsigned long long*)&st->heavy_total, (unsigned long long)chunks);
                    for (int64_t c = 0; c < chunks; ++c) {
                        if (at + c < P.heavy_cap)
                            P.heavy[at + c] = HeavyItem{i, phase, 0, (int32_t)c, q.seg};
                        else
                            set_error(st, DERR_HEAVY_CAPACITY);
                    }
                    m = 0;
                }
            }
        }
        for (int64_t w = 0; __any_sync(kFull, w < m); ++w) {
            WSpawn rec;
            bool sp = false;
            if (w < m) sp = wide_walker(pr, q, w, walker_word(q, w), &rec);
            warp_append(P, W, sp, rec, lane);
        }
    }
}

// ---------------------------------------------------------------------------
// Heavy parents: one warp per work item.  Item c of a parent covers the
// walkers 2 + 4 b + (0..3) of its extra calls b in [c kWChunk, (c + 1)
// kWChunk), one call per lane and round; item 0 also the walkers 0 and 1.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kWThreads) k_wide_heavy(StepParams P, WideParams W)
{
    DevState* st = P.st;
    if (cta_error(st)) return;
    const StepInfo inf = P.info[st->call_index];
    const int64_t items = min((int64_t)st->heavy_total, P.heavy_cap);
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t it = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); it < items; it += warps) {
        const HeavyItem h = P.heavy[it];
        const int slot = h.phase ? (st->cur + 2) % 3 : st->cur;
        WParent q;
        WProg pr;
        if (!load_parent(P, inf, (const WRec*)P.pop[slot], P.segoff[slot], h.parent, h.phase, &q, &pr)) continue;
        const int64_t m = iabs64(q.re) + iabs64(q.im);
        if (h.chunk == 0) {
            WSpawn rec;
            bool sp = false;
            if (lane < 2 && lane < m) sp = wide_walker(pr, q, lane, walker_word(q, lane), &rec);
            warp_append(P, W, sp, rec, lane);
        }
        const int64_t nb = (m - 2 + 3) / 4;   // extra calls of the parent
        const int64_t b0 = (int64_t)h.chunk * kWChunk, b1 = min(nb, b0 + kWChunk);
        for (int64_t bb = b0; bb < b1; bb += 32) {
            const int64_t b = bb + lane;
            uint4 o = make_uint4(0u, 0u, 0u, 0u);
            if (b < b1) o = extra_words(q.rank, (uint32_t)b, h.phase, q.kd);
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const int64_t w = 2 + 4 * b + k;
                WSpawn rec;
                bool sp = false;
                if (b < b1 && w < m) sp = wide_walker(pr, q, w, word_of(o, k), &rec);
                warp_append(P, W, sp, rec, lane);
            }
        }
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
    if (cta_error(P.st)) return;
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
// counts become digit starts.
__global__ void k_wide_plan(StepParams P, WideParams W)
{
    __shared__ uint32_t s_skip;
    if (cta_error(P.st)) return;
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
__device__ __forceinline__ int64_t lower_bound_pop(const WRec* a, int64_t lo, int64_t hi, u128 k)
{
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (wkey(a[mid]) < k) lo = mid + 1; else hi = mid;
    }
    return lo;
}

__device__ __forceinline__ int64_t lower_bound_spawn(const WSpawn* a, int64_t lo, int64_t hi, u128 k)
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

// Runs of equal (vector, key) among the sorted spawns, at their first record.
__global__ void __launch_bounds__(kWThreads) k_wide_runs(StepParams P, WideParams W)
{
    DevState* st = P.st;
    if (cta_error(st)) return;
    const WSpawn* sp = sorted_spawns(W);
    const int64_t S = spawn_count(P);
    const int cur = st->cur;
    const WRec* A = (const WRec*)P.pop[cur];
    const int64_t* offA = P.segoff[cur];
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < S; i += (int64_t)gridDim.x * blockDim.x) {
        const WSpawn r = wsload(sp, i);
        const u128 k = wkey(r);
        const uint32_t seg = r.meta >> 2;
        if (i > 0) {
            const WSpawn q = wsload(sp, i - 1);
            if ((q.meta >> 2) == seg && wkey(q) == k) {
                W.flag_u[i] = 0;
                continue;
            }
        }
        int64_t ire = 0, iim = 0, are = 0, aim = 0;
        for (int64_t j = i; j < S; ++j) {
            const WSpawn q = wsload(sp, j);
            if ((q.meta >> 2) != seg || wkey(q) != k) break;
            const int64_t v = q.val;
            const bool to_im = (q.meta >> 1) & 1u;
            if (to_im) aim += v; else are += v;
            if (!(q.meta & 1u)) {
                if (to_im) iim += v; else ire += v;
            }
        }
        const int64_t lo = offA[seg], hi = offA[seg + 1];
        const int64_t pos = lower_bound_pop(A, lo, hi, k);
        const bool matched = pos < hi && wkey(A[pos]) == k;
        WRun run;
        run.posA = pos;
        run.re = matched ? are : ire;
        run.im = matched ? aim : iim;
        run.matched = matched ? 1 : 0;
        run.pad = 0;
        W.run[i] = run;
        const bool fresh = !matched && (ire != 0 || iim != 0);
        if (fresh && (iabs64(ire) > 2147483647ll || iabs64(iim) > 2147483647ll)) set_error(st, DERR_POP_OVERFLOW);
        W.flag_u[i] = fresh ? 1 : 0;
    }
}

// Each record of N(t) with the spawn run on its key (if any).
__global__ void __launch_bounds__(kWThreads) k_wide_match(StepParams P, WideParams W)
{
    DevState* st = P.st;
    if (cta_error(st)) return;
    const WSpawn* sp = sorted_spawns(W);
    const int cur = st->cur;
    const WRec* A = (const WRec*)P.pop[cur];
    const int64_t* offA = P.segoff[cur];
    const int64_t K = offA[P.nseg];
    int seg = -1;
    int64_t seg_end = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < K; i += (int64_t)gridDim.x * blockDim.x) {
        if (seg < 0 || i >= seg_end || i < offA[seg]) {
            seg = seg_of(offA, P.nseg, i);
            seg_end = offA[seg + 1];
        }
        const WRec a = wload(A, i);
        const u128 k = wkey(a);
        const int64_t lo = P.bseg[seg], hi = P.bseg[seg + 1];
        const int64_t lb = lower_bound_spawn(sp, lo, hi, k);
        int64_t re = a.re, im = a.im;
        if (lb < hi && wkey(sp[lb]) == k) {
            const WRun run = W.run[lb];
            re += run.re;
            im += run.im;
        }
        if (iabs64(re) > 2147483647ll || iabs64(im) > 2147483647ll) {
            set_error(st, DERR_POP_OVERFLOW);
            re = im = 0;
        }
        W.aux[i] = WAux{lb, (int32_t)re, (int32_t)im};
        W.flag_a[i] = (re != 0 || im != 0) ? 1 : 0;
    }
}

// Exclusive prefix sums of 0/1 flags (count n, read from the device):
// per-tile sums, their prefix (one CTA), the tiles' own prefixes; out[n] is
// the total.  which 0: the records of N(t); 1: the spawns.
__device__ __forceinline__ int64_t flag_count(const StepParams& P, int which)
{
    return which ? spawn_count(P) : P.segoff[P.st->cur][P.nseg];
}

__global__ void __launch_bounds__(kWThreads) k_wide_scan_part(StepParams P, WideParams W, int which)
{
    __shared__ int64_t red[kWThreads / 32];
    if (cta_error(P.st)) return;
    const int32_t* f = which ? W.flag_u : W.flag_a;
    const int64_t N = flag_count(P, which);
    const int64_t tiles = (N + kWScanTile - 1) / kWScanTile;
    for (int64_t t = blockIdx.x; t < tiles; t += gridDim.x) {
        int64_t c = 0;
        const int64_t e1 = min(N, (t + 1) * kWScanTile);
        for (int64_t e = t * kWScanTile + threadIdx.x; e < e1; e += blockDim.x) c += f[e];
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

__global__ void __launch_bounds__(kWThreads) k_wide_scan_top(StepParams P, WideParams W, int which)
{
    __shared__ int64_t wsum[kWThreads / 32];
    if (cta_error(P.st)) return;
    const int64_t N = flag_count(P, which);
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
    if (threadIdx.x == 0) {
        int64_t* out = which ? W.scan_u : W.scan_a;
        out[N] = carry;
    }
}

__global__ void __launch_bounds__(kWThreads) k_wide_scan_apply(StepParams P, WideParams W, int which)
{
    constexpr int kPer = kWScanTile / kWThreads;
    __shared__ int64_t wsum[kWThreads / 32];
    if (cta_error(P.st)) return;
    const int32_t* f = which ? W.flag_u : W.flag_a;
    int64_t* out = which ? W.scan_u : W.scan_a;
    const int64_t N = flag_count(P, which);
    const int64_t tiles = (N + kWScanTile - 1) / kWScanTile;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int64_t t = blockIdx.x; t < tiles; t += gridDim.x) {
        // each thread a run of kPer consecutive flags
        const int64_t e0 = t * kWScanTile + (int64_t)threadIdx.x * kPer;
        int v[kPer];
        int c = 0;
#pragma unroll
        for (int k = 0; k < kPer; ++k) {
            v[k] = e0 + k < N ? f[e0 + k] : 0;
            c += v[k];
        }
        int incl = c;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int x = __shfl_up_sync(kFull, incl, o);
            if (lane >= o) incl += x;
        }
        if (lane == 31) wsum[warp] = incl;
        __syncthreads();
        int64_t run = W.part[t];
        for (int q = 0; q < warp; ++q) run += wsum[q];
        run += incl - c;
#pragma unroll
        for (int k = 0; k < kPer; ++k) {
            if (e0 + k < N) out[e0 + k] = run;
            run += v[k];
        }
        __syncthreads();
    }
}

} // namespace

namespace {

// Output offsets of the vectors: survivors of N(t) before vector s plus new
// keys before it.  Raises POP_CAPACITY when N(t + dt) does not fit.
__global__ void k_wide_outoff(StepParams P, WideParams W)
{
    DevState* st = P.st;
    if (cta_error(st)) return;
    const int cur = st->cur, nxt = (cur + 1) % 3;
    const int64_t* offA = P.segoff[cur];
    int64_t* off = P.segoff[nxt];
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s <= P.nseg; s += gridDim.x * blockDim.x)
        off[s] = W.scan_a[offA[s]] + W.scan_u[P.bseg[s]];
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        const int64_t total = W.scan_a[offA[P.nseg]] + W.scan_u[spawn_count(P)];
        st->next_total = total;
        if (total > st->max_next) st->max_next = total;
        if (total > P.pop_cap) set_error(st, DERR_POP_CAPACITY);
    }
}

__global__ void __launch_bounds__(kWThreads) k_wide_scatter_a(StepParams P, WideParams W)
{
    DevState* st = P.st;
    if (cta_error(st)) return;
    const int cur = st->cur;
    const WRec* A = (const WRec*)P.pop[cur];
    WRec* out = (WRec*)P.pop[(cur + 1) % 3];
    const int64_t K = P.segoff[cur][P.nseg];
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < K; i += (int64_t)gridDim.x * blockDim.x) {
        if (!W.flag_a[i]) continue;
        const WAux x = W.aux[i];
        WRec r;
        r.lo = A[i].lo;
        r.hi = A[i].hi;
        r.re = x.re;
        r.im = x.im;
        out[W.scan_a[i] + W.scan_u[x.lbS]] = r;
    }
}

__global__ void __launch_bounds__(kWThreads) k_wide_scatter_u(StepParams P, WideParams W)
{
    DevState* st = P.st;
    if (cta_error(st)) return;
    const int cur = st->cur;
    const WSpawn* sp = sorted_spawns(W);
    WRec* out = (WRec*)P.pop[(cur + 1) % 3];
    const int64_t S = spawn_count(P);
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < S; i += (int64_t)gridDim.x * blockDim.x) {
        if (!W.flag_u[i]) continue;
        const WRun run = W.run[i];
        WRec r;
        r.lo = sp[i].lo;
        r.hi = sp[i].hi;
        r.re = (int32_t)run.re;
        r.im = (int32_t)run.im;
        out[W.scan_u[i] + W.scan_a[run.posA]] = r;
    }
}

// Per-vector K, N_tot and N^diag of a slot: each CTA a contiguous range, a
// thread accumulating while its vector stays the same.
__global__ void __launch_bounds__(kWThreads) k_wide_obs(StepParams P, int slot_rel, SegStats* __restrict__ out)
{
    const DevState* st = P.st;
    if (read_error(st)) return;
    const int slot = (st->cur + slot_rel) % 3;
    const WRec* pop = (const WRec*)P.pop[slot];
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
        st->acc_sort_lsd += 1;
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

void configure_wide_kernels() { (void)wide_grid(); }

// The kernels of one step, in order, on one stream (captured into a graph by
// the host).
void launch_wide_step(const StepParams& P, const WideParams& W, cudaStream_t s)
{
    const int g = wide_grid();
    k_wide_prologue<<<1, kWThreads, 0, s>>>(P);
    k_wide_zero_hist<<<1, kWThreads, 0, s>>>(W);
    k_wide_spawn<<<g, kWThreads, 0, s>>>(P, W, 0);
    k_wide_spawn<<<g, kWThreads, 0, s>>>(P, W, 1);
    k_wide_heavy<<<g, kWThreads, 0, s>>>(P, W);
    k_wide_hist<<<g, kWThreads, 0, s>>>(P, W);
    k_wide_plan<<<1, kWThreads, 0, s>>>(P, W);
    for (int p = 0; p < W.passes; ++p) {
        k_wide_tile_hist<<<g, kWThreads, 0, s>>>(P, W, p);
        k_wide_tile_scan<<<256, kWThreads, 0, s>>>(P, W, p);
        k_wide_scatter<<<g, kWThreads, 0, s>>>(P, W, p);
    }
    k_wide_spawn_off<<<g, kWThreads, 0, s>>>(P, W);
    k_wide_runs<<<g, kWThreads, 0, s>>>(P, W);
    k_wide_match<<<g, kWThreads, 0, s>>>(P, W);
    for (int which = 0; which < 2; ++which) {
        k_wide_scan_part<<<g, kWThreads, 0, s>>>(P, W, which);
        k_wide_scan_top<<<1, kWThreads, 0, s>>>(P, W, which);
        k_wide_scan_apply<<<g, kWThreads, 0, s>>>(P, W, which);
    }
    k_wide_outoff<<<g, kWThreads, 0, s>>>(P, W);
    k_wide_scatter_a<<<g, kWThreads, 0, s>>>(P, W);
    k_wide_scatter_u<<<g, kWThreads, 0, s>>>(P, W);
    k_wide_obs<<<g, kWThreads, 0, s>>>(P, 1, P.segacc);
    k_wide_finalize<<<1, kWThreads, 0, s>>>(P);
}

int wide_step_launch_count(const StepParams& P, const WideParams& W)
{
    (void)P;
    return 7 + 3 * W.passes + 3 + 6 + 5;
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
    WRec* dst = (WRec*)P.pop[slot];
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
            if (keep && pos + excl < P.pop_cap) {
                const u128 k = ((u128)xs[e] << n) | (u128)ys[e];
                WRec r;
                r.lo = (uint64_t)k;
                r.hi = (uint64_t)(k >> 64);
                r.re = (int32_t)vals[2 * i];
                r.im = (int32_t)vals[2 * i + 1];
                dst[pos + excl] = r;
            }
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
    const WRec* A = (const WRec*)P.pop[cur];
    const int64_t lo = P.segoff[cur][seg], hi = P.segoff[cur][seg + 1];
    const int n = P.seginfo[seg].n;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nq; i += gridDim.x * blockDim.x) {
        const u128 k = ((u128)qx[i] << n) | (u128)qy[i];
        const int64_t p = lower_bound_pop(A, lo, hi, k);
        const bool hit = p < hi && wkey(A[p]) == k;
        out[2 * i] = hit ? A[p].re : 0;
        out[2 * i + 1] = hit ? A[p].im : 0;
    }
}

__global__ void k_wide_export(StepParams P, int slot, int64_t first, int64_t count, uint64_t* __restrict__ x,
                              uint64_t* __restrict__ y, int32_t* __restrict__ re, int32_t* __restrict__ im)
{
    const WRec* A = (const WRec*)P.pop[slot];
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x) {
        const WRec r = A[first + i];
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
