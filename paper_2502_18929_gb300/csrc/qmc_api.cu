// C ABI of the library (include/qmc.h): context, memory, step orchestration,
// results, checkpoints.  Kernels live in kernels.cu, the term compiler in
// term_compiler.cpp.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <atomic>
#include <condition_variable>
#include <memory>
#include <mutex>
#include <thread>
#include <vector>
#include <chrono>

#include "../../include/qmc.h"
#include "kernels.h"
#include "wide.h"
#include "qmc_types.h"
#include "term_compiler.h"
#include "context.h"

using namespace qmc;


namespace {

// Records per population slot and spawn records per step: parent indices are
// 32-bit and look-back values 36-bit; 2^31 - 1 keeps every signed 32-bit
// intermediate in range.
constexpr int64_t kLookbackValueLimit = (1ll << 31) - 1;
// Look-back status words carry a 26-bit epoch that advances by 16 per step
// launch; clearing the status arrays at least every 2^20 launches keeps a
// stale word from ever carrying the current epoch.
constexpr int64_t kStatusClearLaunches = (int64_t)1 << 20;

int fail(qmc_ctx* c, int code, const std::string& why)
{
    if (c) c->err = why;
    return code;
}

#define CK(call)                                                                          \
    do {                                                                                  \
        cudaError_t e_ = (call);                                                          \
        if (e_ != cudaSuccess)                                                            \
            return fail(ctx, QMC_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

// Device memory of the context: from the caller's allocator when one was
// given, else from the context's pool, both in stream order on the work
// stream (no device-wide synchronisation when a buffer grows).
void* mem_alloc(qmc_ctx* ctx, size_t bytes)
{
    if (bytes == 0) bytes = 16;
    void* p = nullptr;
    if (ctx->cfg.alloc) {
        p = ctx->cfg.alloc((uint64_t)bytes, (void*)ctx->work, ctx->cfg.alloc_user);
    } else if (cudaMallocFromPoolAsync(&p, bytes, ctx->pool, ctx->work) != cudaSuccess) {
        cudaGetLastError();
        p = nullptr;
    }
    if (p) {
        ctx->blocks[p] = bytes;
        ctx->held_bytes += (int64_t)bytes;
    }
    return p;
}

void mem_free(qmc_ctx* ctx, void* p)
{
    if (!p) return;
    auto it = ctx->blocks.find(p);
    if (it == ctx->blocks.end()) return;   // not ours
    ctx->held_bytes -= (int64_t)it->second;
    ctx->blocks.erase(it);
    if (ctx->cfg.alloc)
        ctx->cfg.free(p, (void*)ctx->work, ctx->cfg.alloc_user);
    else
        cudaFreeAsync(p, ctx->work);
}

template <typename T>
int dalloc(qmc_ctx* ctx, T** p, int64_t count)
{
    mem_free(ctx, *p);
    *p = nullptr;
    if (count <= 0) count = 1;
    *p = (T*)mem_alloc(ctx, (size_t)count * sizeof(T));
    if (!*p) return fail(ctx, QMC_ERR_OOM, "device allocation of " + std::to_string((size_t)count * sizeof(T)) + " bytes failed");
    return QMC_OK;
}

// Temporary device buffers of one call, returned in stream order when the
// call ends, on its error paths too.
struct Scratch {
    qmc_ctx* ctx;
    std::vector<void*> held;
    explicit Scratch(qmc_ctx* c) : ctx(c) {}
    ~Scratch()
    {
        for (void* p : held) mem_free(ctx, p);
    }
    template <typename T>
    int get(T** p, int64_t count)
    {
        *p = (T*)mem_alloc(ctx, (size_t)std::max<int64_t>(count, 1) * sizeof(T));
        if (!*p) return fail(ctx, QMC_ERR_OOM, "no device memory for a temporary buffer");
        held.push_back(*p);
        return QMC_OK;
    }
};

int seg_bits_of(int nseg)
{
    int b = 0;
    while ((1ll << b) < nseg) ++b;
    return b;
}

// Hash of the problem(s) and configuration a checkpoint belongs to.
uint64_t context_hash(const qmc_ctx* c)
{
    if (!c->batch) {
        const qmc_ctx::Instance& I = c->inst[0];
        return schedule_hash(I.sched, I.seed, I.nvec, c->cfg.integrator, I.n_diag, I.init_min);
    }
    uint64_t h = 1469598103934665603ull;
    for (const auto& I : c->inst) {
        const uint64_t v[2] = {schedule_hash(I.sched, I.seed, I.nvec, c->cfg.integrator, I.n_diag, I.init_min),
                               (uint64_t)I.n};
        const uint8_t* b = (const uint8_t*)v;
        for (size_t i = 0; i < sizeof(v); ++i) {
            h ^= b[i];
            h *= 1099511628211ull;
        }
    }
    return h;
}

// The instance that owns segment seg.
const qmc_ctx::Instance& instance_of(const qmc_ctx* c, int seg)
{
    size_t lo = 0, hi = c->inst.size() - 1;
    while (lo < hi) {
        const size_t mid = (lo + hi + 1) / 2;
        if (c->inst[mid].seg0 <= seg) lo = mid; else hi = mid - 1;
    }
    return c->inst[lo];
}

bool has_schedules(const qmc_ctx* c)
{
    for (const auto& I : c->inst)
        if (!I.has_sched) return false;
    return true;
}

StepParams params(qmc_ctx* c)
{
    StepParams P;
    std::memset(&P, 0, sizeof(P));
    P.st = c->d_state;
    P.info = c->d_info;
    P.progs = c->d_progs;
    for (int i = 0; i < 3; ++i) {
        P.pop[i] = c->d_pop[i];
        P.segoff[i] = c->d_segoff[i];
        P.gofs[i] = c->d_gofs[i];
    }
    P.pop_cap = c->pop_cap;
    P.spawn = c->d_spawn;
    P.spawn_alt = c->d_spawn_alt;
    P.spawn_cap = c->spawn_cap;
    P.cand = c->d_cand;
    P.cand_cap = c->cand_cap;
    P.heavy = c->d_heavy;
    P.heavy_cap = c->heavy_cap;
    P.kd = c->d_kd;
    P.sort_hist = c->d_sort_hist;
    P.sort_status = c->d_sort_status;
    P.sort_tiles_cap = c->sort_tiles_cap;
    P.bseg = c->d_bseg;
    P.tile_start = c->d_tile_start;
    P.mtiles = c->d_mtiles;
    P.merge_status = c->d_merge_status;
    P.merge_tiles_cap = c->merge_tiles_cap;
    P.segacc = c->d_segacc;
    P.history = c->d_history;
    P.zacc = c->d_zacc;
    P.zhist = c->d_zhist;
    P.history_cap = c->history_cap;
    P.n = c->cfg.n_qubits;
    P.nseg = c->cfg.n_segments;
    P.seg_bits = seg_bits_of(c->cfg.n_segments);
    P.key_passes = (2 * c->cfg.n_qubits + 7) / 8;
    P.seg_passes = (P.seg_bits + 7) / 8;
    {
        // bucket digit: every segment bit and the top key bits, sized so that
        // a full spawn buffer puts about 24 records in a bucket (10 to
        // kBucketBits bits, never more than the sort key has)
        const int total = P.seg_bits + 2 * c->cfg.n_qubits;
        int want = 10;
        while (want < kBucketBits && ((int64_t)c->bucket_records << want) < c->spawn_cap) ++want;
        if (want < P.seg_bits) want = P.seg_bits;
        P.bucket_bits = total < want ? total : want;
        P.bucket_kb = P.bucket_bits - P.seg_bits;
        // (window sorts keep the vector in 20 bits above a 12-bit index, padding at vector 2^20 - 1)
        P.sort_mode = (P.bucket_bits > kBucketBits || P.seg_bits > 19) ? 0 : (P.bucket_bits == total ? 2 : 1);
        P.bucket = c->d_bucket;
        P.bscan_status = c->d_bscan_status;
        P.big_list = c->d_big_list;
    }
    P.seginfo = c->d_seginfo;
    P.inst = c->d_inst;
    P.ninst = (int)c->inst.size();
    P.proposal = c->proposal;
    P.heavy_walkers = c->heavy_walkers;
    P.spin_limit = c->spin_limit;
    P.mlp = c->d_mlp;
    P.mlp_mask = c->d_mlp_mask;
    P.mlp_idx = c->d_mlp_idx;
    P.mlp_in = c->mlp_in;
    P.mlp_hidden = c->mlp_hidden;
    P.mlp_out = c->mlp_out;
    P.mlp_eps = c->mlp_eps;
    P.mlp_tc = c->d_mlp_tc;
    {
        const TcLayout L = tc_layout(c->mlp_in, c->mlp_hidden, c->mlp_out);
        P.mlp_ip = L.Ip;
        P.mlp_gp = L.Gp;
    }
    return P;
}

WideParams wparams(qmc_ctx* c)
{
    WideParams W;
    std::memset(&W, 0, sizeof(W));
    W.spawn = c->d_wspawn;
    W.spawn_alt = c->d_wspawn_alt;
    W.run = c->d_wrun;
    W.flag_u = c->d_wflag_u;
    W.scan_u = c->d_wscan_u;
    W.delta = c->d_wdelta;
    W.newcnt = c->d_wnewcnt;
    W.mtile = c->d_wmtile;
    W.mbase = c->d_wmbase;
    W.mtiles_cap = c->wmtiles_cap;
    W.abound = c->d_wabound;
    W.win = c->d_wwin;
    W.big_list = c->d_wbig;
    W.nbig = c->d_wnbig;
    W.scan_a = c->d_wscan_a;
    W.part = c->d_wpart;
    W.part_cap = c->wpart_cap;
    W.hist = c->d_whist;
    W.tile_hist = c->d_wtile;
    W.tiles_cap = c->wtiles_cap;
    W.plan = c->d_wplan;
    W.passes = (2 * c->cfg.n_qubits + seg_bits_of(c->cfg.n_segments) + 7) / 8;
    return W;
}

// Make the work stream wait for the caller's stream (and vice versa at exit).
int enter(qmc_ctx* ctx)
{
    CK(cudaSetDevice(ctx->device));
    CK(cudaEventRecord(ctx->ev, ctx->user_stream));
    CK(cudaStreamWaitEvent(ctx->work, ctx->ev, 0));
    return QMC_OK;
}

int leave(qmc_ctx* ctx)
{
    CK(cudaEventRecord(ctx->ev, ctx->work));
    CK(cudaStreamWaitEvent(ctx->user_stream, ctx->ev, 0));
    return QMC_OK;
}

// Account for n step launches about to be issued on the work stream, clearing
// the look-back status arrays first when the epoch could otherwise wrap.
int note_launches(qmc_ctx* ctx, int64_t n)
{
    if (ctx->launches_since_clear + n > kStatusClearLaunches) {
        if (ctx->d_sort_status)
            CK(cudaMemsetAsync(ctx->d_sort_status, 0, (size_t)ctx->sort_tiles_cap * 256 * 8, ctx->work));
        if (ctx->d_merge_status)
            CK(cudaMemsetAsync(ctx->d_merge_status, 0, (size_t)ctx->merge_tiles_cap * 8, ctx->work));
        if (ctx->d_bscan_status)
            CK(cudaMemsetAsync(ctx->d_bscan_status, 0, (size_t)8 << (kBucketBits - 10), ctx->work));
        ctx->launches_since_clear = 0;
    }
    ctx->launches_since_clear += n;
    return QMC_OK;
}

// Prefix-sum partials of the wide step: one per kWScanTile records or spawns.
int grow_wpart(qmc_ctx* ctx)
{
    const int64_t cap = std::max(ctx->pop_cap, ctx->spawn_cap) / kWScanTile + 2;
    if (cap <= ctx->wpart_cap) return QMC_OK;
    int rc;
    if ((rc = dalloc(ctx, &ctx->d_wpart, cap)) != QMC_OK) return rc;
    ctx->wpart_cap = cap;
    ctx->graph_dirty = true;
    return QMC_OK;
}

int grow_spawn(qmc_ctx* ctx, int64_t need)
{
    int64_t cap = std::max<int64_t>(need + need / 2, 1 << 16);
    if (cap > kLookbackValueLimit) cap = kLookbackValueLimit;
    if (need > cap) return fail(ctx, QMC_ERR_CAPACITY, "spawn records exceed 2^31 - 1 per step");
    int rc;
    if (ctx->wide) {
        if ((rc = dalloc(ctx, &ctx->d_wspawn, cap)) != QMC_OK || (rc = dalloc(ctx, &ctx->d_wspawn_alt, cap)) != QMC_OK ||
            (rc = dalloc(ctx, &ctx->d_wrun, cap)) != QMC_OK || (rc = dalloc(ctx, &ctx->d_wflag_u, cap)) != QMC_OK ||
            (rc = dalloc(ctx, &ctx->d_wscan_u, cap + 1)) != QMC_OK)
            return rc;
        ctx->wtiles_cap = (cap + kWTile - 1) / kWTile + 1;
        if ((rc = dalloc(ctx, &ctx->d_wtile, ctx->wtiles_cap * 256)) != QMC_OK) return rc;
        // sort windows of whole buckets: one per 224 spawn records, and those too large for a warp
        if ((rc = dalloc(ctx, &ctx->d_wwin, cap / 224 + 2)) != QMC_OK) return rc;
        if ((rc = dalloc(ctx, &ctx->d_wbig, cap / 224 + 2)) != QMC_OK) return rc;
        ctx->spawn_cap = cap;
        ctx->graph_dirty = true;
        return grow_wpart(ctx);
    }
    if ((rc = dalloc(ctx, &ctx->d_spawn, cap)) != QMC_OK) return rc;
    if ((rc = dalloc(ctx, &ctx->d_spawn_alt, cap)) != QMC_OK) return rc;
    // buckets of more than 32 records, sorted by a CTA each: at most one per 33 spawn records
    if ((rc = dalloc(ctx, &ctx->d_big_list, cap / 32 + 2)) != QMC_OK) return rc;
    ctx->spawn_cap = cap;
    ctx->sort_tiles_cap = (cap + kSortTile - 1) / kSortTile + 1;
    if ((rc = dalloc(ctx, &ctx->d_sort_status, ctx->sort_tiles_cap * 256)) != QMC_OK) return rc;
    CK(cudaMemsetAsync(ctx->d_sort_status, 0, (size_t)ctx->sort_tiles_cap * 256 * 8, ctx->work));
    ctx->graph_dirty = true;
    return QMC_OK;
}

int grow_cand(qmc_ctx* ctx, int64_t need)
{
    const int64_t cap = std::max<int64_t>(need + need / 2, 1 << 16);
    int rc;
    if ((rc = dalloc(ctx, &ctx->d_cand, cap)) != QMC_OK) return rc;
    ctx->cand_cap = cap;
    ctx->graph_dirty = true;
    return QMC_OK;
}

int grow_merge_tiles(qmc_ctx* ctx)
{
    if (ctx->wide) return QMC_OK;   // nor merge tiles
    const int64_t cap = (ctx->pop_cap + ctx->spawn_cap) / kMergeTile + ctx->cfg.n_segments + 2;
    if (cap <= ctx->merge_tiles_cap) return QMC_OK;
    int rc;
    if ((rc = dalloc(ctx, &ctx->d_mtiles, cap)) != QMC_OK) return rc;
    if ((rc = dalloc(ctx, &ctx->d_merge_status, cap)) != QMC_OK) return rc;
    CK(cudaMemsetAsync(ctx->d_merge_status, 0, (size_t)cap * 8, ctx->work));
    ctx->merge_tiles_cap = cap;
    ctx->graph_dirty = true;
    return QMC_OK;
}

// Grow the three population slots to hold need records, keeping contents.
int grow_pop(qmc_ctx* ctx, int64_t need)
{
    int64_t cap = std::max<int64_t>(need + need / 2, 1 << 12);
    if (cap > kLookbackValueLimit) cap = kLookbackValueLimit;
    if (need > cap) return fail(ctx, QMC_ERR_CAPACITY, "population exceeds 2^31 - 1 records");
    if (ctx->cfg.max_records > 0 && need > ctx->cfg.max_records)
        return fail(ctx, QMC_ERR_CAPACITY, "population exceeds max_records");
    if (ctx->cfg.max_records > 0) cap = std::min(cap, ctx->cfg.max_records);
    DevState hs;
    CK(cudaMemcpyAsync(&hs, ctx->d_state, sizeof(hs), cudaMemcpyDeviceToHost, ctx->work));
    CK(cudaStreamSynchronize(ctx->work));
    const size_t rec_bytes = ctx->wide ? sizeof(WRec) : sizeof(Rec);
    for (int i = 0; i < 3; ++i) {
        Rec* np = (Rec*)mem_alloc(ctx, (size_t)cap * rec_bytes);
        if (!np) return fail(ctx, QMC_ERR_OOM, "population buffer allocation failed");
        const int64_t keep = std::min<int64_t>(hs.count[i], std::min(ctx->pop_cap, cap));
        if (ctx->d_pop[i] && keep > 0 && ctx->wide) {
            // keys [0, cap) x 16 bytes, then values x 8 bytes: the value region moves with the capacity
            uint8_t* dst = (uint8_t*)np;
            const uint8_t* src = (const uint8_t*)ctx->d_pop[i];
            CK(cudaMemcpyAsync(dst, src, (size_t)keep * 16, cudaMemcpyDeviceToDevice, ctx->work));
            CK(cudaMemcpyAsync(dst + 16 * (size_t)cap, src + 16 * (size_t)ctx->pop_cap, (size_t)keep * 8,
                               cudaMemcpyDeviceToDevice, ctx->work));
        } else if (ctx->d_pop[i] && keep > 0) {
            CK(cudaMemcpyAsync(np, ctx->d_pop[i], (size_t)keep * rec_bytes, cudaMemcpyDeviceToDevice, ctx->work));
        }
        mem_free(ctx, ctx->d_pop[i]);   // in stream order, after the copy
        ctx->d_pop[i] = np;
    }
    ctx->pop_cap = cap;
    ctx->graph_dirty = true;
    if (ctx->wide) {
        int rc;
        if ((rc = dalloc(ctx, &ctx->d_wdelta, cap + 1)) != QMC_OK ||
            (rc = dalloc(ctx, &ctx->d_wnewcnt, cap + 1)) != QMC_OK ||
            (rc = dalloc(ctx, &ctx->d_wscan_a, cap + 2)) != QMC_OK)
            return rc;
        ctx->wmtiles_cap = cap / kWMTile + 2;
        if ((rc = dalloc(ctx, &ctx->d_wmtile, ctx->wmtiles_cap)) != QMC_OK ||
            (rc = dalloc(ctx, &ctx->d_wmbase, ctx->wmtiles_cap)) != QMC_OK)
            return rc;
        CK(cudaMemsetAsync(ctx->d_wdelta, 0, (size_t)(cap + 1) * sizeof(int2), ctx->work));
        CK(cudaMemsetAsync(ctx->d_wnewcnt, 0, (size_t)(cap + 1) * sizeof(int32_t), ctx->work));
        CK(cudaMemsetAsync(ctx->d_wmtile, 0, (size_t)ctx->wmtiles_cap * 8, ctx->work));
        return grow_wpart(ctx);
    }
    return grow_merge_tiles(ctx);
}

// Host threads building column programs, over every context of the process:
// concurrent step calls share the cores instead of taking up to 16 each.
std::atomic<int> g_builders{0};

// Builder threads for a call that wants `want`: what the process has left
// (hardware threads less those building), at least one.
int reserve_builders(int want)
{
    const unsigned hw = std::thread::hardware_concurrency();
    const int cap = (int)(hw ? hw : 1);
    int cur = g_builders.load();
    for (;;) {
        const int take = std::max(1, std::min(want, cap - cur));
        if (g_builders.compare_exchange_weak(cur, cur + take)) return take;
    }
}

// Step table and history of a qmc_step call of nsteps steps: device and
// pinned staging capacity (before any of its steps is launched).
int ensure_call_capacity(qmc_ctx* ctx, int64_t nsteps)
{
    int rc;
    if (nsteps > ctx->info_cap) {
        if ((rc = dalloc(ctx, &ctx->d_info, nsteps)) != QMC_OK) return rc;
        ctx->info_cap = nsteps;
        ctx->graph_dirty = true;
    }
    if (nsteps > ctx->history_cap) {
        if ((rc = dalloc(ctx, &ctx->d_history, nsteps * ctx->cfg.n_segments)) != QMC_OK) return rc;
        if ((rc = dalloc(ctx, &ctx->d_zhist, nsteps * ctx->cfg.n_segments * ctx->cfg.n_qubits)) != QMC_OK) return rc;
        ctx->history_cap = nsteps;
        ctx->graph_dirty = true;
    }
    if (nsteps > ctx->h_info_cap) {
        CK(cudaStreamSynchronize(ctx->work));   // no copy from the old staging is pending
        if (ctx->h_info) cudaFreeHost(ctx->h_info);
        ctx->h_info = nullptr;
        ctx->h_info_cap = 0;
        if (cudaMallocHost((void**)&ctx->h_info, (size_t)nsteps * sizeof(StepInfo)) != cudaSuccess)
            return fail(ctx, QMC_ERR_OOM, "pinned staging of the step table failed");
        ctx->h_info_cap = nsteps;
    }
    return QMC_OK;
}

// Program space of a call (bytes), device and pinned staging.  A new device
// buffer holds nothing: the caller uploads the programs again.
int ensure_progs(qmc_ctx* ctx, int64_t bytes)
{
    int rc;
    if (bytes > ctx->progs_cap) {
        if ((rc = dalloc(ctx, &ctx->d_progs, bytes)) != QMC_OK) return rc;
        ctx->progs_cap = bytes;
        ctx->graph_dirty = true;
    }
    if (bytes > ctx->h_progs_cap) {
        CK(cudaStreamSynchronize(ctx->work));   // no copy from the old staging is pending
        if (ctx->h_progs) cudaFreeHost(ctx->h_progs);
        ctx->h_progs = nullptr;
        ctx->h_progs_cap = 0;
        if (cudaMallocHost((void**)&ctx->h_progs, (size_t)bytes) != cudaSuccess)
            return fail(ctx, QMC_ERR_OOM, "pinned staging of the column programs failed");
        ctx->h_progs_cap = bytes;
    }
    return QMC_OK;
}

int capture_graph(qmc_ctx* ctx)
{
    if (!ctx->graph_dirty && ctx->graph) return QMC_OK;
    if (ctx->graph) {
        cudaGraphExecDestroy(ctx->graph);
        ctx->graph = nullptr;
    }
    StepParams P = params(ctx);
    cudaGraph_t g;
    CK(cudaStreamBeginCapture(ctx->work, cudaStreamCaptureModeThreadLocal));
    if (ctx->wide)
        launch_wide_step(P, wparams(ctx), ctx->work);
    else
        launch_step(P, ctx->grid, ctx->work);
    CK(cudaStreamEndCapture(ctx->work, &g));
    cudaError_t e = cudaGraphInstantiate(&ctx->graph, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return fail(ctx, QMC_ERR_CUDA, std::string("cudaGraphInstantiate: ") + cudaGetErrorString(e));
    ctx->graph_dirty = false;
    return QMC_OK;
}

int map_dev_error(qmc_ctx* ctx, uint32_t code, uint32_t aux = 0)
{
    char site[64];
    std::snprintf(site, sizeof(site), " (wait site %u, index %u)", aux >> 24, aux & 0xFFFFFFu);
    switch (code) {
    case DERR_DT_TOO_LARGE: return fail(ctx, QMC_ERR_DT_TOO_LARGE, "spawn probability p >= 1: reduce dt");
    case DERR_POP_OVERFLOW: return fail(ctx, QMC_ERR_POP_OVERFLOW, "a population component exceeds 2^31 - 1");
    case DERR_TIMEOUT: return fail(ctx, QMC_ERR_DEVICE_TIMEOUT, std::string("a bounded device wait expired") + site);
    case DERR_INTERNAL: return fail(ctx, QMC_ERR_STATE, "the step's self-check failed: merge counts disagree");
    default: return fail(ctx, QMC_ERR_CAPACITY, "capacity error");
    }
}

int clear_dev_error(qmc_ctx* ctx)
{
    const uint32_t zero = 0;
    CK(cudaMemcpyAsync((uint8_t*)ctx->d_state + offsetof(DevState, error), &zero, sizeof(zero),
                       cudaMemcpyHostToDevice, ctx->work));
    CK(cudaStreamSynchronize(ctx->work));
    return QMC_OK;
}

} // namespace

extern "C" {

} // extern "C"

namespace {

// Shared by qmc_create and qmc_batch_create: cfg carries the totals
// (n_qubits = largest instance, n_segments = all vectors); inst the instances.
int create_context(qmc_ctx** out, const qmc_config* cfg, std::vector<qmc_ctx::Instance>&& inst, bool batch)
{
    qmc_ctx* ctx = new qmc_ctx();
    ctx->cfg = *cfg;
    ctx->inst = std::move(inst);
    ctx->batch = batch;
    ctx->wide = cfg->n_qubits > 32;
    ctx->user_stream = (cudaStream_t)cfg->cuda_stream;
    int rc = QMC_OK;
    auto bail = [&](int code) { qmc_destroy(ctx); return code; };
    if (cudaGetDevice(&ctx->device) != cudaSuccess) return bail(QMC_ERR_CUDA);
    cudaDeviceGetAttribute(&ctx->sm_count, cudaDevAttrMultiProcessorCount, ctx->device);
    ctx->grid = cfg->max_ctas > 0 ? cfg->max_ctas : 0;   // 0: each kernel fills the GPU
    configure_kernels();
    configure_wide_kernels();
    if (cudaStreamCreateWithFlags(&ctx->work, cudaStreamNonBlocking) != cudaSuccess) return bail(QMC_ERR_CUDA);
    if (cudaEventCreateWithFlags(&ctx->ev, cudaEventDisableTiming) != cudaSuccess) return bail(QMC_ERR_CUDA);
    if ((cfg->alloc == nullptr) != (cfg->free == nullptr)) return bail(QMC_ERR_INVALID_ARG);
    if (!cfg->alloc) {
        cudaMemPoolProps props{};
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = ctx->device;
        if (cudaMemPoolCreate(&ctx->pool, &props) != cudaSuccess) return bail(QMC_ERR_CUDA);
        uint64_t keep_all = ~0ull;   // freed blocks stay in the pool for the next growth
        cudaMemPoolSetAttribute(ctx->pool, cudaMemPoolAttrReleaseThreshold, &keep_all);
    }
    const int nseg = cfg->n_segments;
    if ((rc = dalloc(ctx, &ctx->d_state, 1)) != QMC_OK) return bail(rc);
    if (cudaMemsetAsync(ctx->d_state, 0, sizeof(DevState), ctx->work) != cudaSuccess) return bail(QMC_ERR_CUDA);
    for (int i = 0; i < 3; ++i) {
        if ((rc = dalloc(ctx, &ctx->d_segoff[i], nseg + 1)) != QMC_OK) return bail(rc);
        if ((rc = dalloc(ctx, &ctx->d_gofs[i], nseg + 1)) != QMC_OK) return bail(rc);
        if (cudaMemsetAsync(ctx->d_segoff[i], 0, (size_t)(nseg + 1) * 8, ctx->work) != cudaSuccess)
            return bail(QMC_ERR_CUDA);
    }
    if ((rc = dalloc(ctx, &ctx->d_kd, nseg)) != QMC_OK) return bail(rc);
    if ((rc = dalloc(ctx, &ctx->d_bucket, (int64_t)1 << kBucketBits)) != QMC_OK) return bail(rc);
    if ((rc = dalloc(ctx, &ctx->d_bscan_status, (int64_t)1 << (kBucketBits - 10))) != QMC_OK) return bail(rc);
    if (cudaMemsetAsync(ctx->d_bscan_status, 0, (size_t)8 << (kBucketBits - 10), ctx->work) != cudaSuccess)
        return bail(QMC_ERR_CUDA);
    if ((rc = dalloc(ctx, &ctx->d_sort_hist, kMaxPasses * 256)) != QMC_OK) return bail(rc);
    if ((rc = dalloc(ctx, &ctx->d_bseg, nseg + 1)) != QMC_OK) return bail(rc);
    if ((rc = dalloc(ctx, &ctx->d_tile_start, nseg + 1)) != QMC_OK) return bail(rc);
    if ((rc = dalloc(ctx, &ctx->d_segacc, nseg)) != QMC_OK) return bail(rc);
    if ((rc = dalloc(ctx, &ctx->d_zacc, 32 * (int64_t)nseg)) != QMC_OK) return bail(rc);
    if ((rc = dalloc(ctx, &ctx->d_obs, nseg)) != QMC_OK) return bail(rc);
    // heavy work items: at most one per 64 records of the hinted capacity to start with
    ctx->heavy_cap = std::max<int64_t>(4096, cfg->capacity_hint / 64);
    if ((rc = dalloc(ctx, &ctx->d_heavy, ctx->heavy_cap)) != QMC_OK) return bail(rc);
    if (ctx->wide && ((rc = dalloc(ctx, &ctx->d_whist, kWMaxPasses * 256)) != QMC_OK ||
                      (rc = dalloc(ctx, &ctx->d_wnbig, 1)) != QMC_OK ||
                      (rc = dalloc(ctx, &ctx->d_wplan, kWMaxPasses + 1)) != QMC_OK ||
                      (rc = dalloc(ctx, &ctx->d_wabound, ((int64_t)1 << kBucketBits) + 1)) != QMC_OK))
        return bail(rc);
    const int64_t hint = cfg->capacity_hint > 0 ? cfg->capacity_hint : (int64_t)1 << 16;
    if ((rc = grow_spawn(ctx, hint / 4 + 1024)) != QMC_OK) return bail(rc);
    if ((rc = grow_cand(ctx, hint / 4 + 1024)) != QMC_OK) return bail(rc);
    if ((rc = grow_pop(ctx, hint)) != QMC_OK) return bail(rc);
    {
        // segment and instance tables
        std::vector<SegInfo> si(nseg);
        std::vector<InstInfo> ii(ctx->inst.size());
        for (size_t i = 0; i < ctx->inst.size(); ++i) {
            const qmc_ctx::Instance& I = ctx->inst[i];
            ii[i] = InstInfo{I.seed, I.n_diag, I.init_min, I.n, I.nvec};
            for (int v = 0; v < I.nvec; ++v) si[I.seg0 + v] = SegInfo{(int32_t)i, I.n, v, 0};
        }
        if ((rc = dalloc(ctx, &ctx->d_seginfo, nseg)) != QMC_OK) return bail(rc);
        if ((rc = dalloc(ctx, &ctx->d_inst, (int64_t)ii.size())) != QMC_OK) return bail(rc);
        if (cudaMemcpyAsync(ctx->d_seginfo, si.data(), si.size() * sizeof(SegInfo), cudaMemcpyHostToDevice,
                            ctx->work) != cudaSuccess ||
            cudaMemcpyAsync(ctx->d_inst, ii.data(), ii.size() * sizeof(InstInfo), cudaMemcpyHostToDevice,
                            ctx->work) != cudaSuccess ||
            cudaStreamSynchronize(ctx->work) != cudaSuccess)
            return bail(QMC_ERR_CUDA);
    }
    if (cudaStreamSynchronize(ctx->work) != cudaSuccess) return bail(QMC_ERR_CUDA);
    *out = ctx;
    return QMC_OK;
}

} // namespace

extern "C" {

int qmc_create(qmc_ctx** out, const qmc_config* cfg)
{
    if (!out || !cfg) return QMC_ERR_INVALID_ARG;
    if (cfg->n_qubits < 1 || cfg->n_qubits > QMC_MAX_QUBITS || cfg->n_segments < 1 || cfg->n_diag < 1 ||
        cfg->n_segments > (1 << 28) || (cfg->integrator != QMC_EULER && cfg->integrator != QMC_AB2) ||
        cfg->initiator_min < 0)
        return QMC_ERR_INVALID_ARG;
    std::vector<qmc_ctx::Instance> inst(1);
    inst[0].n = cfg->n_qubits;
    inst[0].nvec = cfg->n_segments;
    inst[0].seg0 = 0;
    inst[0].seed = cfg->seed;
    inst[0].n_diag = cfg->n_diag;
    inst[0].init_min = cfg->initiator_min;
    return create_context(out, cfg, std::move(inst), false);
}

int qmc_batch_create(qmc_ctx** out, const qmc_instance* inst, int32_t n_instances, const qmc_config* cfg)
{
    if (!out || !inst || !cfg || n_instances < 1) return QMC_ERR_INVALID_ARG;
    if (cfg->integrator != QMC_EULER && cfg->integrator != QMC_AB2) return QMC_ERR_INVALID_ARG;
    std::vector<qmc_ctx::Instance> v((size_t)n_instances);
    int64_t nseg = 0;
    int nmax = 0;
    for (int i = 0; i < n_instances; ++i) {
        const qmc_instance& q = inst[i];
        if (q.n_qubits < 1 || q.n_qubits > 32 || q.n_vectors < 1 || q.n_diag < 1 || q.initiator_min < 0)
            return QMC_ERR_INVALID_ARG;
        if (q.n_ham < 0 || q.n_lind < 0 || q.n_coefs < 0 || q.n_rates < 0 || q.n_windows < 0 ||
            (q.n_ham && !q.ham) || (q.n_lind && !q.lind) || (q.n_coefs && !q.coefs) || (q.n_rates && !q.rates) ||
            (q.n_windows && !q.windows))
            return QMC_ERR_INVALID_ARG;
        qmc_ctx::Instance& I = v[i];
        I.n = q.n_qubits;
        I.nvec = q.n_vectors;
        I.seg0 = (int32_t)nseg;
        I.seed = q.seed;
        I.n_diag = q.n_diag;
        I.init_min = q.initiator_min;
        I.sched.n = q.n_qubits;
        I.sched.ham.assign(q.ham, q.ham + q.n_ham);
        I.sched.lind.assign(q.lind, q.lind + q.n_lind);
        I.sched.coefs.assign(q.coefs, q.coefs + q.n_coefs);
        I.sched.rates.assign(q.rates, q.rates + q.n_rates);
        I.sched.windows.assign(q.windows, q.windows + q.n_windows);
        std::string why;
        if (validate_schedule(I.sched, &why) != QMC_OK) return QMC_ERR_INVALID_ARG;
        I.has_sched = true;
        nseg += q.n_vectors;
        nmax = std::max(nmax, q.n_qubits);
        if (nseg > (1 << 28)) return QMC_ERR_INVALID_ARG;
    }
    qmc_config c = *cfg;
    c.n_qubits = nmax;
    c.n_segments = (int32_t)nseg;
    c.seed = 0;
    c.n_diag = 1;
    c.initiator_min = 0;
    return create_context(out, &c, std::move(v), true);
}

void qmc_destroy(qmc_ctx* ctx)
{
    if (!ctx) return;
    if (ctx->work) cudaStreamSynchronize(ctx->work);
    if (ctx->graph) cudaGraphExecDestroy(ctx->graph);
    std::vector<void*> held;
    for (const auto& b : ctx->blocks) held.push_back(b.first);
    for (void* p : held) mem_free(ctx, p);
    if (ctx->work) cudaStreamSynchronize(ctx->work);
    if (ctx->h_info) cudaFreeHost(ctx->h_info);
    if (ctx->h_progs) cudaFreeHost(ctx->h_progs);
    if (ctx->pool) cudaMemPoolDestroy(ctx->pool);
    if (ctx->ev) cudaEventDestroy(ctx->ev);
    if (ctx->work) cudaStreamDestroy(ctx->work);
    delete ctx;
}

int qmc_memory(const qmc_ctx* ctx, int64_t* out)
{
    if (!ctx || !out) return QMC_ERR_INVALID_ARG;
    out[0] = ctx->held_bytes;
    out[1] = (int64_t)ctx->blocks.size();
    return QMC_OK;
}

const char* qmc_last_error(const qmc_ctx* ctx)
{
    if (!ctx) return "null context";
    return ctx->err.c_str();
}

int qmc_load_schedule(qmc_ctx* ctx, const qmc_ham_term* ham, int32_t n_ham, const qmc_lindblad* lind,
                      int32_t n_lind, const qmc_pauli_coef* coefs, int32_t n_coefs, const qmc_rate* rates,
                      int32_t n_rates, const qmc_window* windows, int32_t n_windows)
{
    if (!ctx) return QMC_ERR_INVALID_ARG;
    if (ctx->batch) return fail(ctx, QMC_ERR_STATE, "a batch takes its schedules at qmc_batch_create");
    if (n_ham < 0 || n_lind < 0 || n_coefs < 0 || n_rates < 0 || n_windows < 0)
        return fail(ctx, QMC_ERR_INVALID_ARG, "negative array length");
    Schedule s;
    s.n = ctx->cfg.n_qubits;
    if (n_ham) s.ham.assign(ham, ham + n_ham);
    if (n_lind) s.lind.assign(lind, lind + n_lind);
    if (n_coefs) s.coefs.assign(coefs, coefs + n_coefs);
    if (n_rates) s.rates.assign(rates, rates + n_rates);
    if (n_windows) s.windows.assign(windows, windows + n_windows);
    std::string why;
    if (validate_schedule(s, &why) != QMC_OK) return fail(ctx, QMC_ERR_INVALID_ARG, why);
    ctx->inst[0].sched = s;
    ctx->inst[0].has_sched = true;
    return QMC_OK;
}

namespace {
// The network in the tensor-core proposal's layout (bf16 weights), rebuilt
// from the fp32 parameters whenever they change; left null when the network
// does not fit that path (hidden width a multiple of 16 up to 64, at most 256
// outputs and 80 inputs).
int repack_tc(qmc_ctx* ctx)
{
    const int I = ctx->mlp_in, H = ctx->mlp_hidden, G = ctx->mlp_out;
    if (!ctx->d_mlp || H % 16 != 0 || H > 64 || G > 256 || I > 80) {
        mem_free(ctx, ctx->d_mlp_tc);
        ctx->d_mlp_tc = nullptr;
        return QMC_OK;
    }
    const TcLayout L = tc_layout(I, H, G);
    int rc;
    if ((rc = dalloc(ctx, &ctx->d_mlp_tc, (int64_t)L.bytes)) != QMC_OK) return rc;
    launch_mlp_tc_pack(ctx->d_mlp, L, ctx->d_mlp_tc, ctx->work);
    CK(cudaGetLastError());
    return QMC_OK;
}
} // namespace

int qmc_set_proposal(qmc_ctx* ctx, int32_t kind)
{
    if (ctx && ctx->wide && kind != QMC_PROPOSAL_EXACT)
        return fail(ctx, QMC_ERR_INVALID_ARG, "only the exact spawn choice above 32 qubits");
    if (!ctx) return QMC_ERR_INVALID_ARG;
    if (kind != QMC_PROPOSAL_EXACT && kind != QMC_PROPOSAL_STATIC && kind != QMC_PROPOSAL_LEARNED &&
        kind != QMC_PROPOSAL_LEARNED_TC)
        return fail(ctx, QMC_ERR_INVALID_ARG, "unknown proposal kind");
    if ((kind == QMC_PROPOSAL_LEARNED || kind == QMC_PROPOSAL_LEARNED_TC) && !ctx->d_mlp)
        return fail(ctx, QMC_ERR_STATE, "load the learned proposal's network first");
    if (kind == QMC_PROPOSAL_LEARNED_TC && !ctx->d_mlp_tc)
        return fail(ctx, QMC_ERR_INVALID_ARG,
                    "the tensor-core proposal needs a hidden width of 16, 32, 48 or 64, at most 256 outputs and 80 inputs");
    if (ctx->proposal != kind) {
        ctx->proposal = kind;
        ctx->graph_dirty = true;
    }
    return QMC_OK;
}

int qmc_set_proposal_mlp(qmc_ctx* ctx, const qmc_mlp* m)
{
    if (ctx && ctx->wide) return fail(ctx, QMC_ERR_INVALID_ARG, "qmc_set_proposal_mlp: not available above 32 qubits");
    if (!ctx || !m) return QMC_ERR_INVALID_ARG;
    if (ctx->batch) return fail(ctx, QMC_ERR_STATE, "the learned proposal takes a context of one instance");
    const int n = ctx->inst[0].n, I = m->n_in, H = m->n_hidden, G = m->n_out;
    if (I != 2 * n + 1 || H < 1 || H > 64 || G < 1 || G > 4096 || !(m->eps > 0.0f) || m->eps > 1.0f ||
        !m->out_masks || !m->w1 || !m->b1 || !m->w2 || !m->b2 || !m->w3 || !m->b3)
        return fail(ctx, QMC_ERR_INVALID_ARG, "network sizes or pointers out of range");
    std::vector<std::pair<uint64_t, int32_t>> order(G);
    for (int g = 0; g < G; ++g) order[g] = {m->out_masks[g], g};
    std::sort(order.begin(), order.end());
    for (int g = 1; g < G; ++g)
        if (order[g].first == order[g - 1].first) return fail(ctx, QMC_ERR_INVALID_ARG, "output masks repeat");
    std::vector<uint64_t> masks(G);
    std::vector<int32_t> idx(G);
    for (int g = 0; g < G; ++g) {
        masks[g] = order[g].first;
        idx[g] = order[g].second;
    }
    std::vector<float> w;
    w.insert(w.end(), m->w1, m->w1 + (size_t)H * I);
    w.insert(w.end(), m->b1, m->b1 + H);
    w.insert(w.end(), m->w2, m->w2 + (size_t)H * H);
    w.insert(w.end(), m->b2, m->b2 + H);
    w.insert(w.end(), m->w3, m->w3 + (size_t)G * H);
    w.insert(w.end(), m->b3, m->b3 + G);
    int rc;
    if ((rc = enter(ctx)) != QMC_OK) return rc;
    if ((rc = dalloc(ctx, &ctx->d_mlp, (int64_t)w.size())) != QMC_OK) return rc;
    if ((rc = dalloc(ctx, &ctx->d_mlp_mask, G)) != QMC_OK) return rc;
    if ((rc = dalloc(ctx, &ctx->d_mlp_idx, G)) != QMC_OK) return rc;
    CK(cudaMemcpyAsync(ctx->d_mlp, w.data(), w.size() * 4, cudaMemcpyHostToDevice, ctx->work));
    CK(cudaMemcpyAsync(ctx->d_mlp_mask, masks.data(), (size_t)G * 8, cudaMemcpyHostToDevice, ctx->work));
    CK(cudaMemcpyAsync(ctx->d_mlp_idx, idx.data(), (size_t)G * 4, cudaMemcpyHostToDevice, ctx->work));
    CK(cudaStreamSynchronize(ctx->work));
    ctx->mlp_in = I;
    ctx->mlp_hidden = H;
    ctx->mlp_out = G;
    ctx->mlp_eps = m->eps;
    if ((rc = repack_tc(ctx)) != QMC_OK) return rc;
    if (ctx->proposal == QMC_PROPOSAL_LEARNED_TC && !ctx->d_mlp_tc) ctx->proposal = QMC_PROPOSAL_EXACT;
    ctx->graph_dirty = true;
    return leave(ctx);
}

namespace {
int64_t mlp_param_count(const qmc_ctx* c)
{
    const int64_t I = c->mlp_in, H = c->mlp_hidden, G = c->mlp_out;
    return H * I + H + H * H + H + G * H + G;
}
} // namespace


int qmc_learned_weights(qmc_ctx* ctx, double t, double dt_eff, const uint64_t* x, const uint64_t* y, int32_t count,
                        int64_t* Q, int32_t cap_slots, int32_t* n_slots)
{
    if (ctx && ctx->wide) return fail(ctx, QMC_ERR_INVALID_ARG, "qmc_learned_weights: not available above 32 qubits");
    if (!ctx || !n_slots || count < 0 || cap_slots < 0 || (count > 0 && (!x || !y || !Q)) || !(dt_eff > 0.0))
        return QMC_ERR_INVALID_ARG;
    const bool tc = ctx->proposal == QMC_PROPOSAL_LEARNED_TC;
    if (!tc && ctx->proposal != QMC_PROPOSAL_LEARNED)
        return fail(ctx, QMC_ERR_INVALID_ARG, "qmc_learned_weights: set a learned proposal first");
    if (!has_schedules(ctx) || !ctx->d_mlp || (tc && !ctx->d_mlp_tc))
        return fail(ctx, QMC_ERR_STATE, "load a schedule and the network first");
    const int n = ctx->inst[0].n;
    const uint64_t lim = (1ull << n) - 1ull;
    for (int32_t i = 0; i < count; ++i)
        if ((x[i] & ~lim) || (y[i] & ~lim)) return fail(ctx, QMC_ERR_INVALID_ARG, "x or y >= 2^n");
    std::vector<uint8_t> blob;
    int rc = build_program(ctx->inst[0].sched, t, dt_eff, &blob);
    if (rc != QMC_OK) return fail(ctx, rc, "coefficient * rate * dt >= 2^10");
    const ProgHeader* h = (const ProgHeader*)blob.data();
    *n_slots = h->n_stat;
    if (h->n_stat > kMaxLearnedSlots) return fail(ctx, QMC_ERR_INVALID_ARG, "more than 256 destinations per column");
    if (h->n_stat > cap_slots) return fail(ctx, QMC_ERR_INVALID_ARG, "cap_slots below the column's slot count");
    if (count == 0) return QMC_OK;
    if ((rc = enter(ctx)) != QMC_OK) return rc;
    uint8_t* d_prog = nullptr;
    uint64_t *d_x = nullptr, *d_y = nullptr;
    int64_t* d_q = nullptr;
    Scratch tmp(ctx);
    if ((rc = tmp.get(&d_prog, (int64_t)blob.size())) != QMC_OK || (rc = tmp.get(&d_x, count)) != QMC_OK ||
        (rc = tmp.get(&d_y, count)) != QMC_OK || (rc = tmp.get(&d_q, (int64_t)count * h->n_stat)) != QMC_OK)
        return rc;
    CK(cudaMemcpyAsync(d_prog, blob.data(), blob.size(), cudaMemcpyHostToDevice, ctx->work));
    CK(cudaMemcpyAsync(d_x, x, (size_t)count * 8, cudaMemcpyHostToDevice, ctx->work));
    CK(cudaMemcpyAsync(d_y, y, (size_t)count * 8, cudaMemcpyHostToDevice, ctx->work));
    launch_learned_weights(params(ctx), tc, d_prog, t, d_x, d_y, count, d_q, h->n_stat, ctx->work);
    CK(cudaGetLastError());
    std::vector<int64_t> hq((size_t)count * h->n_stat);
    CK(cudaMemcpyAsync(hq.data(), d_q, hq.size() * 8, cudaMemcpyDeviceToHost, ctx->work));
    CK(cudaStreamSynchronize(ctx->work));
    for (int32_t i = 0; i < count; ++i)
        for (int k = 0; k < h->n_stat; ++k) Q[(int64_t)i * cap_slots + k] = hq[(size_t)i * h->n_stat + k];
    return leave(ctx);
}

int qmc_learn_param_count(qmc_ctx* ctx, int64_t* n_params)
{
    if (!ctx || !n_params) return QMC_ERR_INVALID_ARG;
    if (!ctx->d_mlp) return fail(ctx, QMC_ERR_STATE, "load the learned proposal's network first");
    *n_params = mlp_param_count(ctx);
    return QMC_OK;
}

int qmc_learn_events(qmc_ctx* ctx, double dt, int64_t max_events, float* feat, float* target, float* weight,
                     int64_t* n_events)
{
    if (ctx && ctx->wide) return fail(ctx, QMC_ERR_INVALID_ARG, "qmc_learn_events: not available above 32 qubits");
    if (!ctx || !feat || !target || !weight || !n_events) return QMC_ERR_INVALID_ARG;
    if (!ctx->d_mlp) return fail(ctx, QMC_ERR_STATE, "load the learned proposal's network first");
    if (!has_schedules(ctx) || !ctx->has_pop) return fail(ctx, QMC_ERR_STATE, "load a schedule and populations first");
    if (!(dt > 0.0) || max_events < 1) return fail(ctx, QMC_ERR_INVALID_ARG, "dt must be > 0 and max_events >= 1");
    std::vector<uint8_t> blob;
    int rc = build_program(ctx->inst[0].sched, ctx->t, dt, &blob);
    if (rc == QMC_ERR_COEF_RANGE) return fail(ctx, rc, "coefficient * rate * dt >= 2^10");
    if (rc != QMC_OK) return rc;
    if ((rc = enter(ctx)) != QMC_OK) return rc;
    if ((int64_t)blob.size() > ctx->learn_prog_cap) {
        if ((rc = dalloc(ctx, &ctx->d_learn_prog, (int64_t)blob.size())) != QMC_OK) return rc;
        ctx->learn_prog_cap = (int64_t)blob.size();
    }
    if (!ctx->d_learn_small && (rc = dalloc(ctx, &ctx->d_learn_small, 4)) != QMC_OK) return rc;
    CK(cudaMemcpyAsync(ctx->d_learn_prog, blob.data(), blob.size(), cudaMemcpyHostToDevice, ctx->work));
    LearnArgs A;
    A.st = ctx->d_state;
    for (int s = 0; s < 3; ++s) A.pop[s] = ctx->d_pop[s];
    A.prog = ctx->d_learn_prog;
    A.masks = ctx->d_mlp_mask;
    A.idx = ctx->d_mlp_idx;
    A.n = ctx->inst[0].n;
    A.G = ctx->mlp_out;
    A.t = ctx->t;
    A.max_events = max_events;
    A.ld = max_events;
    A.feat = feat;
    A.target = target;
    A.weight = weight;
    A.n_events = (int64_t*)ctx->d_learn_small;
    launch_learn_events(A, ctx->work);
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(n_events, ctx->d_learn_small, 8, cudaMemcpyDeviceToHost, ctx->work));
    CK(cudaStreamSynchronize(ctx->work));
    return leave(ctx);
}

int qmc_learn_grad(qmc_ctx* ctx, const float* params, const float* feat, const float* target, const float* weight,
                   int64_t ld, int64_t n_events, float* grad, double* loss)
{
    if (ctx && ctx->wide) return fail(ctx, QMC_ERR_INVALID_ARG, "qmc_learn_grad: not available above 32 qubits");
    if (!ctx || !params || !feat || !target || !weight || !grad || !loss) return QMC_ERR_INVALID_ARG;
    if (!ctx->d_mlp) return fail(ctx, QMC_ERR_STATE, "load the learned proposal's network first");
    if (n_events < 1 || ld < n_events) return fail(ctx, QMC_ERR_INVALID_ARG, "need 1 <= n_events <= ld");
    const int64_t H = ctx->mlp_hidden, G = ctx->mlp_out;
    const int64_t rows = 4 * H + G + 1;
    if (rows * ld > ((int64_t)1 << 28)) return fail(ctx, QMC_ERR_INVALID_ARG, "events x (4 hidden + outputs) above 2^28");
    int rc;
    if ((rc = enter(ctx)) != QMC_OK) return rc;
    if (rows * ld > ctx->learn_scratch_cap) {
        if ((rc = dalloc(ctx, &ctx->d_learn_scratch, rows * ld)) != QMC_OK) return rc;
        ctx->learn_scratch_cap = rows * ld;
    }
    if (!ctx->d_learn_small && (rc = dalloc(ctx, &ctx->d_learn_small, 4)) != QMC_OK) return rc;
    LearnGrad A;
    A.params = params;
    A.feat = feat;
    A.target = target;
    A.weight = weight;
    A.ld = ld;
    A.E = n_events;
    A.I = ctx->mlp_in;
    A.H = (int)H;
    A.G = (int)G;
    float* s = ctx->d_learn_scratch;
    A.h1t = s;
    A.h2t = s + H * ld;
    A.d2t = s + 2 * H * ld;
    A.d1t = s + 3 * H * ld;
    A.dzt = s + 4 * H * ld;
    A.lossv = s + (4 * H + G) * ld;
    A.wsum = ctx->d_learn_small + 1;
    launch_learn_grad(A, grad, ctx->d_learn_small + 2, ctx->work);
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(loss, ctx->d_learn_small + 2, 8, cudaMemcpyDeviceToHost, ctx->work));
    CK(cudaStreamSynchronize(ctx->work));
    return leave(ctx);
}

int qmc_learn_grad_tc(qmc_ctx* ctx, const float* params, const float* feat, const float* target, const float* weight,
                      int64_t ld, int64_t n_events, float* grad, double* loss)
{
    if (ctx && ctx->wide) return fail(ctx, QMC_ERR_INVALID_ARG, "qmc_learn_grad_tc: not available above 32 qubits");
    if (!ctx || !params || !feat || !target || !weight || !grad || !loss) return QMC_ERR_INVALID_ARG;
    if (!ctx->d_mlp) return fail(ctx, QMC_ERR_STATE, "load the learned proposal's network first");
    if (!ctx->d_mlp_tc)
        return fail(ctx, QMC_ERR_INVALID_ARG,
                    "the tensor-core network needs 16, 32, 48 or 64 hidden units, at most 256 outputs and 80 inputs");
    if (n_events < 1 || ld < n_events) return fail(ctx, QMC_ERR_INVALID_ARG, "need 1 <= n_events <= ld");
    if (((uintptr_t)feat & 15u) || ((uintptr_t)target & 15u) || ((uintptr_t)weight & 15u))
        return fail(ctx, QMC_ERR_INVALID_ARG, "event arrays must be 16-byte aligned");
    const int I = ctx->mlp_in, H = ctx->mlp_hidden, G = ctx->mlp_out;
    const int64_t wb = learn_tc_weights_bytes(I, H, G);
    const int64_t need = wb + learn_tc_scratch_bytes(I, H, G, n_events);
    int rc;
    if ((rc = enter(ctx)) != QMC_OK) return rc;
    if (need > ctx->learn_tc_cap) {
        if ((rc = dalloc(ctx, &ctx->d_learn_tc, need)) != QMC_OK) return rc;
        ctx->learn_tc_cap = need;
    }
    if (!ctx->d_learn_small && (rc = dalloc(ctx, &ctx->d_learn_small, 4)) != QMC_OK) return rc;
    const TcLayout L = tc_layout(I, H, G);
    LearnTc A;
    A.params = params;
    A.feat = feat;
    A.target = target;
    A.weight = weight;
    A.ld = ld;
    A.E = n_events;
    A.I = I;
    A.H = H;
    A.G = G;
    A.wts = ctx->d_learn_tc;
    A.ldp = (n_events + 15) / 16 * 16;
    uint8_t* p = ctx->d_learn_tc + (wb + 255) / 256 * 256;
    auto take = [&](int64_t bytes) {
        uint8_t* r = p;
        p += (bytes + 255) / 256 * 256;
        return r;
    };
    A.h1t = (uint16_t*)take(2 * A.ldp * H);
    A.h2t = (uint16_t*)take(2 * A.ldp * H);
    A.d1t = (uint16_t*)take(2 * A.ldp * H);
    A.d2t = (uint16_t*)take(2 * A.ldp * H);
    A.dzt = (uint16_t*)take(2 * A.ldp * L.Gp);
    A.lossv = (float*)take(4 * A.ldp);
    A.partials = (float*)p;
    A.wsum = ctx->d_learn_small + 1;
    launch_learn_grad_tc(A, grad, ctx->d_learn_small + 2, ctx->work);
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(loss, ctx->d_learn_small + 2, 8, cudaMemcpyDeviceToHost, ctx->work));
    CK(cudaStreamSynchronize(ctx->work));
    return leave(ctx);
}

int qmc_learn_adam(qmc_ctx* ctx, float* params, const float* grad, float* m, float* v, int64_t n_params, int64_t t,
                   float lr, float beta1, float beta2, float eps)
{
    if (!ctx || !params || !grad || !m || !v) return QMC_ERR_INVALID_ARG;
    if (!ctx->d_mlp) return fail(ctx, QMC_ERR_STATE, "load the learned proposal's network first");
    if (n_params != mlp_param_count(ctx) || t < 1 || !(lr > 0.0f) || !(beta1 >= 0.0f && beta1 < 1.0f) ||
        !(beta2 >= 0.0f && beta2 < 1.0f) || !(eps > 0.0f))
        return fail(ctx, QMC_ERR_INVALID_ARG, "Adam: parameter count or hyperparameters out of range");
    int rc;
    if ((rc = enter(ctx)) != QMC_OK) return rc;
    launch_learn_adam(params, grad, m, v, n_params, t, lr, beta1, beta2, eps, ctx->work);
    CK(cudaGetLastError());
    return leave(ctx);
}

int qmc_learn_load(qmc_ctx* ctx, const float* params)
{
    if (!ctx || !params) return QMC_ERR_INVALID_ARG;
    if (!ctx->d_mlp) return fail(ctx, QMC_ERR_STATE, "load the learned proposal's network first");
    int rc;
    if ((rc = enter(ctx)) != QMC_OK) return rc;
    CK(cudaMemcpyAsync(ctx->d_mlp, params, (size_t)mlp_param_count(ctx) * 4, cudaMemcpyDeviceToDevice, ctx->work));
    if (ctx->d_mlp_tc) launch_mlp_tc_pack(ctx->d_mlp, tc_layout(ctx->mlp_in, ctx->mlp_hidden, ctx->mlp_out),
                                          ctx->d_mlp_tc, ctx->work);
    CK(cudaGetLastError());
    return leave(ctx);
}

int qmc_set_tuning(qmc_ctx* ctx, const qmc_tuning* t)
{
    if (!ctx || !t) return QMC_ERR_INVALID_ARG;
    if (t->max_ctas < 0 || t->heavy_walkers < 16 || t->heavy_walkers > (1 << 20) || t->bucket_records < 4 ||
        t->bucket_records > 256)
        return fail(ctx, QMC_ERR_INVALID_ARG, "launch shapes out of range");
    ctx->grid = t->max_ctas;
    ctx->heavy_walkers = t->heavy_walkers;
    ctx->bucket_records = t->bucket_records;
    ctx->graph_dirty = true;
    return QMC_OK;
}

int qmc_set_spin_limit(qmc_ctx* ctx, uint32_t polls)
{
    if (!ctx) return QMC_ERR_INVALID_ARG;
    if (polls > ((uint32_t)1 << 30)) return fail(ctx, QMC_ERR_INVALID_ARG, "spin limit above 2^30 polls");
    ctx->spin_limit = polls;
    ctx->graph_dirty = true;
    return QMC_OK;
}

int qmc_get_tuning(const qmc_ctx* ctx, qmc_tuning* t)
{
    if (!ctx || !t) return QMC_ERR_INVALID_ARG;
    t->max_ctas = ctx->grid;
    t->heavy_walkers = ctx->heavy_walkers;
    t->bucket_records = ctx->bucket_records;
    t->pad = 0;
    return QMC_OK;
}

int qmc_autotune(qmc_ctx* ctx, double dt, int32_t nsteps, qmc_tuning* out)
{
    if (ctx && ctx->wide) return fail(ctx, QMC_ERR_INVALID_ARG, "qmc_autotune: not available above 32 qubits");
    if (!ctx) return QMC_ERR_INVALID_ARG;
    if (!has_schedules(ctx) || !ctx->has_pop) return fail(ctx, QMC_ERR_STATE, "load a schedule and populations first");
    if (!(dt > 0.0) || nsteps < 1 || nsteps > 64) return fail(ctx, QMC_ERR_INVALID_ARG, "dt must be > 0, 1 <= nsteps <= 64");
    int rc;
    if ((rc = enter(ctx)) != QMC_OK) return rc;
    // snapshot of N(t), N(t - dt), their offsets, the device state and the clock
    DevState hs0;
    CK(cudaMemcpyAsync(&hs0, ctx->d_state, sizeof(hs0), cudaMemcpyDeviceToHost, ctx->work));
    CK(cudaStreamSynchronize(ctx->work));
    const int nseg = ctx->cfg.n_segments;
    const int slot[2] = {hs0.cur, (hs0.cur + 2) % 3};
    Rec* keep[2] = {nullptr, nullptr};
    int64_t* keep_off[2] = {nullptr, nullptr};
    Scratch tmp(ctx);
    for (int w = 0; w < 2; ++w) {
        const int64_t cnt = hs0.count[slot[w]];
        if (tmp.get(&keep[w], cnt) != QMC_OK || tmp.get(&keep_off[w], nseg + 1) != QMC_OK)
            return fail(ctx, QMC_ERR_OOM, "autotune: no room for a copy of the populations");
        if (cnt) CK(cudaMemcpyAsync(keep[w], ctx->d_pop[slot[w]], cnt * sizeof(Rec), cudaMemcpyDeviceToDevice, ctx->work));
        CK(cudaMemcpyAsync(keep_off[w], ctx->d_segoff[slot[w]], (size_t)(nseg + 1) * 8, cudaMemcpyDeviceToDevice,
                           ctx->work));
    }
    const uint64_t step0 = ctx->step;
    const double t0 = ctx->t, tp0 = ctx->t_prev, dl0 = ctx->dt_last;
    const bool pv0 = ctx->prev_valid;
    auto restore = [&]() -> int {
        // buffers may have grown (new pointers, larger capacity) during a trial
        for (int w = 0; w < 2; ++w) {
            const int64_t cnt = hs0.count[slot[w]];
            if (cnt) CK(cudaMemcpyAsync(ctx->d_pop[slot[w]], keep[w], cnt * sizeof(Rec), cudaMemcpyDeviceToDevice,
                                        ctx->work));
            CK(cudaMemcpyAsync(ctx->d_segoff[slot[w]], keep_off[w], (size_t)(nseg + 1) * 8, cudaMemcpyDeviceToDevice,
                               ctx->work));
        }
        DevState now;
        CK(cudaMemcpyAsync(&now, ctx->d_state, sizeof(now), cudaMemcpyDeviceToHost, ctx->work));
        CK(cudaStreamSynchronize(ctx->work));
        DevState back = hs0;
        back.seq = now.seq;   // look-back epochs only move forward
        back.error = 0;
        CK(cudaMemcpyAsync(ctx->d_state, &back, sizeof(back), cudaMemcpyHostToDevice, ctx->work));
        CK(cudaStreamSynchronize(ctx->work));
        ctx->step = step0;
        ctx->t = t0;
        ctx->t_prev = tp0;
        ctx->dt_last = dl0;
        ctx->prev_valid = pv0;
        return QMC_OK;
    };
    qmc_tuning best;
    qmc_get_tuning(ctx, &best);
    auto trial = [&](const qmc_tuning& tu, double* ms) -> int {
        int r;
        if ((r = qmc_set_tuning(ctx, &tu)) != QMC_OK) return r;
        if ((r = restore()) != QMC_OK) return r;
        if ((r = capture_graph(ctx)) != QMC_OK) return r;   // not part of the timed steps
        CK(cudaStreamSynchronize(ctx->work));
        const auto a = std::chrono::steady_clock::now();
        r = qmc_step(ctx, dt, nsteps);
        if (r == QMC_OK) CK(cudaStreamSynchronize(ctx->work));
        const auto b = std::chrono::steady_clock::now();
        *ms = r == QMC_OK ? std::chrono::duration<double, std::milli>(b - a).count() : 1e300;
        return QMC_OK;
    };
    int dev = 0, sms = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    double best_ms = 0.0;
    // the first trial also builds the step graph and warms the caches: time it twice
    if ((rc = trial(best, &best_ms)) != QMC_OK || (rc = trial(best, &best_ms)) != QMC_OK) return rc;
    const int32_t ctas[3] = {0, 2 * sms, sms};
    const int32_t heavy[3] = {64, 256, 1024};
    const int32_t bucket[3] = {12, 24, 48};
    for (int knob = 0; knob < 3 && rc == QMC_OK; ++knob) {
        for (int v = 0; v < 3 && rc == QMC_OK; ++v) {
            qmc_tuning cand = best;
            int32_t* field = knob == 0 ? &cand.max_ctas : (knob == 1 ? &cand.heavy_walkers : &cand.bucket_records);
            const int32_t value = knob == 0 ? ctas[v] : (knob == 1 ? heavy[v] : bucket[v]);
            if (*field == value) continue;
            *field = value;
            double ms = 0.0;
            if ((rc = trial(cand, &ms)) != QMC_OK) break;
            if (ms < 0.98 * best_ms) {
                best = cand;
                best_ms = ms;
            }
        }
    }
    if (rc == QMC_OK) rc = qmc_set_tuning(ctx, &best);
    if (rc == QMC_OK) rc = restore();
    if (rc != QMC_OK) return rc;
    if (out) *out = best;
    return leave(ctx);
}

int qmc_init_populations(qmc_ctx* ctx, const uint64_t* x, const uint64_t* y, const double* re,
                         const double* im, int64_t nnz)
{
    if (!ctx) return QMC_ERR_INVALID_ARG;
    if (!has_schedules(ctx)) return fail(ctx, QMC_ERR_STATE, "load a schedule first");
    if (nnz < 0 || (nnz > 0 && (!x || !y || !re || !im))) return fail(ctx, QMC_ERR_INVALID_ARG, "bad arrays");
    // every instance takes the same rho(0); (x, y) must fit the smallest one
    int nmin = QMC_MAX_QUBITS;
    for (const auto& I : ctx->inst) nmin = std::min(nmin, (int)I.n);
    const uint64_t lim = (1ull << nmin) - 1;
    std::vector<std::pair<std::pair<uint64_t, uint64_t>, int64_t>> order;
    for (int64_t i = 0; i < nnz; ++i) {
        if ((x[i] & ~lim) || (y[i] & ~lim)) return fail(ctx, QMC_ERR_INVALID_ARG, "x or y >= 2^n");
        order.push_back({{x[i], y[i]}, i});
    }
    // (x, y) lexicographic = key order (x << n) | y for every n that holds them
    std::sort(order.begin(), order.end());
    for (size_t i = 1; i < order.size(); ++i)
        if (order[i].first == order[i - 1].first) return fail(ctx, QMC_ERR_INVALID_ARG, "duplicate (x, y)");
    std::vector<uint64_t> hx(nnz), hy(nnz);
    std::vector<double> hre(nnz), him(nnz);
    for (int64_t i = 0; i < nnz; ++i) {
        hx[i] = order[i].first.first;
        hy[i] = order[i].first.second;
        hre[i] = re[order[i].second];
        him[i] = im[order[i].second];
    }
    int rc;
    if ((rc = enter(ctx)) != QMC_OK) return rc;
    const int64_t need = std::max<int64_t>(1, nnz) * ctx->cfg.n_segments;
    if (need > ctx->pop_cap && (rc = grow_pop(ctx, need)) != QMC_OK) return rc;
    uint64_t *d_x = nullptr, *d_y = nullptr;
    double *d_re = nullptr, *d_im = nullptr;
    int64_t* d_vals = nullptr;
    Scratch tmp(ctx);
    if ((rc = tmp.get(&d_x, nnz)) != QMC_OK || (rc = tmp.get(&d_y, nnz)) != QMC_OK ||
        (rc = tmp.get(&d_re, nnz)) != QMC_OK || (rc = tmp.get(&d_im, nnz)) != QMC_OK ||
        (rc = tmp.get(&d_vals, 2 * need)) != QMC_OK)
        return rc;
    DevState hs;
    std::memset(&hs, 0, sizeof(hs));
    CK(cudaMemcpyAsync(ctx->d_state, &hs, sizeof(hs), cudaMemcpyHostToDevice, ctx->work));
    if (nnz) {
        CK(cudaMemcpyAsync(d_x, hx.data(), nnz * 8, cudaMemcpyHostToDevice, ctx->work));
        CK(cudaMemcpyAsync(d_y, hy.data(), nnz * 8, cudaMemcpyHostToDevice, ctx->work));
        CK(cudaMemcpyAsync(d_re, hre.data(), nnz * 8, cudaMemcpyHostToDevice, ctx->work));
        CK(cudaMemcpyAsync(d_im, him.data(), nnz * 8, cudaMemcpyHostToDevice, ctx->work));
    }
    StepParams P = params(ctx);
    if (ctx->wide)
        launch_wide_init(P, d_x, d_y, d_re, d_im, nnz, d_vals, ctx->work);
    else
        launch_init(P, d_x, d_y, d_re, d_im, nnz, d_vals, ctx->work);
    CK(cudaGetLastError());
    CK(cudaMemsetAsync(ctx->d_segoff[2], 0, (size_t)(ctx->cfg.n_segments + 1) * 8, ctx->work));
    CK(cudaMemcpyAsync(&hs, ctx->d_state, sizeof(hs), cudaMemcpyDeviceToHost, ctx->work));
    CK(cudaStreamSynchronize(ctx->work));
    if (hs.error) {
        clear_dev_error(ctx);
        return map_dev_error(ctx, hs.error, hs.error_aux);
    }
    ctx->step = 0;
    ctx->t = ctx->t_prev = ctx->dt_last = 0.0;
    ctx->prev_valid = false;
    ctx->has_pop = true;
    return leave(ctx);
}

int qmc_set_populations(qmc_ctx* ctx, int32_t which, const int64_t* counts, const uint64_t* keys,
                        const int32_t* re, const int32_t* im)
{
    if (ctx && ctx->wide) return fail(ctx, QMC_ERR_INVALID_ARG, "qmc_set_populations: not available above 32 qubits");
    if (!ctx || (which != 0 && which != 1) || !counts) return QMC_ERR_INVALID_ARG;
    const int nseg = ctx->cfg.n_segments;
    std::vector<int64_t> off(nseg + 1, 0);
    for (int s = 0; s < nseg; ++s) {
        if (counts[s] < 0) return fail(ctx, QMC_ERR_INVALID_ARG, "negative count");
        off[s + 1] = off[s] + counts[s];
    }
    const int64_t total = off[nseg];
    if (total > 0 && (!keys || !re || !im)) return fail(ctx, QMC_ERR_INVALID_ARG, "null arrays");
    int rc;
    if ((rc = enter(ctx)) != QMC_OK) return rc;
    if (total > ctx->pop_cap && (rc = grow_pop(ctx, total)) != QMC_OK) return rc;
    DevState hs;
    CK(cudaMemcpyAsync(&hs, ctx->d_state, sizeof(hs), cudaMemcpyDeviceToHost, ctx->work));
    CK(cudaStreamSynchronize(ctx->work));
    const int slot = which == 0 ? hs.cur : (hs.cur + 2) % 3;
    // upload the caller's arrays as they are (pinned memory copies at full
    // link speed), then pack and check on the device
    uint64_t* d_keys = nullptr;
    int32_t *d_re = nullptr, *d_im = nullptr;
    int* d_bad = nullptr;
    Scratch tmp(ctx);
    if ((rc = tmp.get(&d_keys, total)) != QMC_OK || (rc = tmp.get(&d_re, total)) != QMC_OK ||
        (rc = tmp.get(&d_im, total)) != QMC_OK || (rc = tmp.get(&d_bad, 1)) != QMC_OK)
        return rc;
    CK(cudaMemsetAsync(d_bad, 0, sizeof(int), ctx->work));
    if (total) {
        CK(cudaMemcpyAsync(d_keys, keys, total * 8, cudaMemcpyHostToDevice, ctx->work));
        CK(cudaMemcpyAsync(d_re, re, total * 4, cudaMemcpyHostToDevice, ctx->work));
        CK(cudaMemcpyAsync(d_im, im, total * 4, cudaMemcpyHostToDevice, ctx->work));
    }
    CK(cudaMemcpyAsync(ctx->d_segoff[slot], off.data(), (nseg + 1) * 8, cudaMemcpyHostToDevice, ctx->work));
    if (total) launch_pack(d_keys, d_re, d_im, ctx->d_segoff[slot], nseg, ctx->d_seginfo, ctx->d_pop[slot], d_bad,
                           ctx->work);
    CK(cudaGetLastError());
    int bad = 0;
    CK(cudaMemcpyAsync(&bad, d_bad, sizeof(int), cudaMemcpyDeviceToHost, ctx->work));
    CK(cudaStreamSynchronize(ctx->work));
    if (bad) {
        // leave the slot empty rather than half-valid
        std::vector<int64_t> zero(nseg + 1, 0);
        CK(cudaMemcpyAsync(ctx->d_segoff[slot], zero.data(), (nseg + 1) * 8, cudaMemcpyHostToDevice, ctx->work));
        hs.count[slot] = 0;
        CK(cudaMemcpyAsync(ctx->d_state, &hs, sizeof(hs), cudaMemcpyHostToDevice, ctx->work));
        CK(cudaStreamSynchronize(ctx->work));
        return fail(ctx, QMC_ERR_INVALID_ARG,
                    "records must be nonzero, keys < 2^(2n) and strictly ascending within each vector");
    }
    hs.count[slot] = total;
    hs.error = 0;
    CK(cudaMemcpyAsync(ctx->d_state, &hs, sizeof(hs), cudaMemcpyHostToDevice, ctx->work));
    CK(cudaStreamSynchronize(ctx->work));
    if (which == 0) ctx->has_pop = true;
    return leave(ctx);
}

int qmc_set_populations_xy(qmc_ctx* ctx, int32_t which, const int64_t* counts, const uint64_t* x,
                           const uint64_t* y, const int32_t* re, const int32_t* im)
{
    if (!ctx || (which != 0 && which != 1) || !counts) return QMC_ERR_INVALID_ARG;
    const int nseg = ctx->cfg.n_segments;
    std::vector<int64_t> off(nseg + 1, 0);
    for (int s = 0; s < nseg; ++s) {
        if (counts[s] < 0) return fail(ctx, QMC_ERR_INVALID_ARG, "negative count");
        off[s + 1] = off[s] + counts[s];
    }
    const int64_t total = off[nseg];
    if (total > 0 && (!x || !y || !re || !im)) return fail(ctx, QMC_ERR_INVALID_ARG, "null arrays");
    if (!ctx->wide) {
        // 64-bit keys: (x << n) | y per vector, then the key-based call
        std::vector<uint64_t> keys((size_t)std::max<int64_t>(total, 1));
        for (int s = 0; s < nseg; ++s) {
            const int n = instance_of(ctx, s).n;
            const uint64_t lim = (1ull << n) - 1ull;
            for (int64_t i = off[s]; i < off[s + 1]; ++i) {
                if ((x[i] & ~lim) || (y[i] & ~lim)) return fail(ctx, QMC_ERR_INVALID_ARG, "x or y >= 2^n");
                keys[i] = (x[i] << n) | y[i];
            }
        }
        return qmc_set_populations(ctx, which, counts, keys.data(), re, im);
    }
    int rc;
    if ((rc = enter(ctx)) != QMC_OK) return rc;
    if (total > ctx->pop_cap && (rc = grow_pop(ctx, total)) != QMC_OK) return rc;
    DevState hs;
    CK(cudaMemcpyAsync(&hs, ctx->d_state, sizeof(hs), cudaMemcpyDeviceToHost, ctx->work));
    CK(cudaStreamSynchronize(ctx->work));
    const int slot = which == 0 ? hs.cur : (hs.cur + 2) % 3;
    uint64_t *d_x = nullptr, *d_y = nullptr;
    int32_t *d_re = nullptr, *d_im = nullptr;
    int* d_bad = nullptr;
    Scratch tmp(ctx);
    if ((rc = tmp.get(&d_x, total)) != QMC_OK || (rc = tmp.get(&d_y, total)) != QMC_OK ||
        (rc = tmp.get(&d_re, total)) != QMC_OK || (rc = tmp.get(&d_im, total)) != QMC_OK ||
        (rc = tmp.get(&d_bad, 1)) != QMC_OK)
        return rc;
    CK(cudaMemsetAsync(d_bad, 0, sizeof(int), ctx->work));
    if (total) {
        CK(cudaMemcpyAsync(d_x, x, total * 8, cudaMemcpyHostToDevice, ctx->work));
        CK(cudaMemcpyAsync(d_y, y, total * 8, cudaMemcpyHostToDevice, ctx->work));
        CK(cudaMemcpyAsync(d_re, re, total * 4, cudaMemcpyHostToDevice, ctx->work));
        CK(cudaMemcpyAsync(d_im, im, total * 4, cudaMemcpyHostToDevice, ctx->work));
    }
    CK(cudaMemcpyAsync(ctx->d_segoff[slot], off.data(), (nseg + 1) * 8, cudaMemcpyHostToDevice, ctx->work));
    if (total)
        launch_wide_pack(d_x, d_y, d_re, d_im, ctx->d_segoff[slot], nseg, ctx->d_seginfo, (uint8_t*)ctx->d_pop[slot],
                         ctx->pop_cap, d_bad, ctx->work);
    CK(cudaGetLastError());
    int bad = 0;
    CK(cudaMemcpyAsync(&bad, d_bad, sizeof(int), cudaMemcpyDeviceToHost, ctx->work));
    CK(cudaStreamSynchronize(ctx->work));
    if (bad) {
        std::vector<int64_t> zero(nseg + 1, 0);
        CK(cudaMemcpyAsync(ctx->d_segoff[slot], zero.data(), (nseg + 1) * 8, cudaMemcpyHostToDevice, ctx->work));
        hs.count[slot] = 0;
        CK(cudaMemcpyAsync(ctx->d_state, &hs, sizeof(hs), cudaMemcpyHostToDevice, ctx->work));
        CK(cudaStreamSynchronize(ctx->work));
        return fail(ctx, QMC_ERR_INVALID_ARG,
                    "records must be nonzero, x, y < 2^n and (x, y) strictly ascending within each vector");
    }
    hs.count[slot] = total;
    hs.error = 0;
    CK(cudaMemcpyAsync(ctx->d_state, &hs, sizeof(hs), cudaMemcpyHostToDevice, ctx->work));
    CK(cudaStreamSynchronize(ctx->work));
    if (which == 0) ctx->has_pop = true;
    return leave(ctx);
}

int qmc_set_clock(qmc_ctx* ctx, uint64_t step, double t, double t_prev, double dt_last, int32_t prev_valid)
{
    if (!ctx) return QMC_ERR_INVALID_ARG;
    int rc;
    if ((rc = enter(ctx)) != QMC_OK) return rc;
    CK(cudaMemcpyAsync((uint8_t*)ctx->d_state + offsetof(DevState, step), &step, 8, cudaMemcpyHostToDevice,
                       ctx->work));
    CK(cudaStreamSynchronize(ctx->work));
    ctx->step = step;
    ctx->t = t;
    ctx->t_prev = t_prev;
    ctx->dt_last = dt_last;
    ctx->prev_valid = prev_valid != 0;
    return leave(ctx);
}

int qmc_get_clock(const qmc_ctx* ctx, uint64_t* step, double* t, double* t_prev, double* dt_last,
                  int32_t* prev_valid)
{
    if (!ctx) return QMC_ERR_INVALID_ARG;
    if (step) *step = ctx->step;
    if (t) *t = ctx->t;
    if (t_prev) *t_prev = ctx->t_prev;
    if (dt_last) *dt_last = ctx->dt_last;
    if (prev_valid) *prev_valid = ctx->prev_valid ? 1 : 0;
    return QMC_OK;
}

int qmc_spawn_prob_bound(const qmc_ctx* ctx, double t, double dt, double* p_bound)
{
    if (!ctx || !p_bound || !has_schedules(ctx)) return QMC_ERR_INVALID_ARG;
    double b = 0.0;
    for (const auto& I : ctx->inst) b = std::max(b, spawn_prob_bound(I.sched, t, dt * 1.5));
    *p_bound = b;
    return QMC_OK;
}

int qmc_step(qmc_ctx* ctx, double dt, int64_t nsteps)
{
    if (!ctx) return QMC_ERR_INVALID_ARG;
    if (!has_schedules(ctx) || !ctx->has_pop) return fail(ctx, QMC_ERR_STATE, "load a schedule and populations first");
    if (!(dt > 0.0) || nsteps < 0) return fail(ctx, QMC_ERR_INVALID_ARG, "dt must be > 0 and nsteps >= 0");
    if (nsteps == 0) return QMC_OK;
    // per-step column programs of every instance (identical consecutive
    // programs of an instance and pass are shared), and per step a table of
    // their offsets
    const int ni = (int)ctx->inst.size();
    std::vector<StepInfo> info(nsteps);
    std::vector<uint8_t> blob;
    std::vector<int64_t> last_off(2 * (size_t)ni, -1);
    std::vector<std::vector<uint8_t>> last_blob(2 * (size_t)ni);
    struct Job {
        int k, pass;
        double t, dte;
    };
    std::vector<Job> jobs;
    std::vector<int64_t> job0(nsteps + 1);
    const double t0 = ctx->t;
    for (int64_t i = 0; i < nsteps; ++i) {
        const double ti = t0 + (double)i * dt;
        const bool ab2 = ctx->cfg.integrator == QMC_AB2 && (i > 0 || (ctx->prev_valid && ctx->dt_last == dt));
        const double tp = i > 0 ? t0 + (double)(i - 1) * dt : ctx->t_prev;
        info[i].ab2 = ab2 ? 1 : 0;
        info[i].t[0] = ti;
        info[i].t[1] = ab2 ? tp : ti;
        job0[i] = (int64_t)jobs.size();
        for (int k = 0; k < ni; ++k) {
            jobs.push_back(Job{k, 0, ti, ab2 ? dt * 1.5 : dt});
            if (ab2) jobs.push_back(Job{k, 1, tp, dt * 0.5});
        }
    }
    job0[nsteps] = (int64_t)jobs.size();
    // Every (step, instance, pass) program is built by host threads in step
    // order while the GPU runs the steps already built: chunks of 1, 2, 4, ...
    // steps are assembled, copied and launched as soon as their programs are
    // ready, so that building overlaps the device's work.
    const int64_t nj = (int64_t)jobs.size();
    std::vector<std::vector<uint8_t>> built(nj);
    std::vector<int> built_rc(nj, QMC_OK);
    std::unique_ptr<std::atomic<int>[]> ready(new std::atomic<int>[nj]);
    for (int64_t j = 0; j < nj; ++j) ready[j].store(0);
    std::atomic<int64_t> next_job{0};
    std::mutex mu;
    std::condition_variable cv;
    struct Pool {   // joins the builders on every exit path and returns them to the process
        std::vector<std::thread> th;
        std::atomic<int64_t>* next;
        int64_t nj;
        int reserved;
        ~Pool()
        {
            next->store(nj);
            for (auto& t : th) t.join();
            g_builders -= reserved;
        }
    } pool{{}, &next_job, nj, 0};
    {
        const int nthr = reserve_builders((int)std::min<int64_t>(16, nj));
        pool.reserved = nthr;
        for (int w = 0; w < nthr; ++w)
            pool.th.emplace_back([&]() {
                for (;;) {
                    const int64_t j = next_job.fetch_add(1);
                    if (j >= nj) return;
                    built_rc[j] = build_program(ctx->inst[jobs[j].k].sched, jobs[j].t, jobs[j].dte, &built[j]);
                    {
                        std::lock_guard<std::mutex> g(mu);
                        ready[j].store(1);
                    }
                    cv.notify_all();
                }
            });
    }
    int64_t jready = 0;
    auto wait_built = [&](int64_t jend) {
        std::unique_lock<std::mutex> lk(mu);
        cv.wait(lk, [&] {
            while (jready < jend && ready[jready].load()) ++jready;
            return jready >= jend;
        });
    };
    auto add_prog = [&](int64_t j, int64_t* off_out) -> int {
        if (built_rc[j] != QMC_OK) {
            if (built_rc[j] == QMC_ERR_COEF_RANGE) return fail(ctx, built_rc[j], "coefficient * rate * dt >= 2^10");
            return built_rc[j];
        }
        const std::vector<uint8_t>& tmp = built[j];
        const ProgHeader* h = (const ProgHeader*)tmp.data();
        if (h->n_entry > kMaxEntries)
            return fail(ctx, QMC_ERR_INVALID_ARG, "column has more destinations than the heavy path holds");
        if ((ctx->proposal == QMC_PROPOSAL_LEARNED || ctx->proposal == QMC_PROPOSAL_LEARNED_TC) &&
            h->n_stat > kMaxLearnedSlots)
            return fail(ctx, QMC_ERR_INVALID_ARG, "learned proposal: more than 256 destinations per column");
        const size_t slot = 2 * (size_t)jobs[j].k + jobs[j].pass;
        if (last_off[slot] >= 0 && last_blob[slot] == tmp) {
            *off_out = last_off[slot];
            return QMC_OK;
        }
        const size_t at = (blob.size() + 15) & ~(size_t)15;
        blob.resize(at);
        blob.insert(blob.end(), tmp.begin(), tmp.end());
        last_blob[slot] = tmp;
        last_off[slot] = (int64_t)at;
        *off_out = (int64_t)at;
        return QMC_OK;
    };
    int rc;
    if ((rc = enter(ctx)) != QMC_OK) return rc;
    if ((rc = ensure_call_capacity(ctx, nsteps)) != QMC_OK) return rc;
    int32_t zero = 0;
    CK(cudaMemcpyAsync((uint8_t*)ctx->d_state + offsetof(DevState, call_index), &zero, 4, cudaMemcpyHostToDevice,
                       ctx->work));
    // A program that cannot be built stops the call before its step: the
    // steps before it run to completion, then the call returns the error.
    int build_err = QMC_OK;
    int64_t nrun = 0;   // steps assembled and launched
    int64_t uploaded = 0;
    std::vector<int64_t> tab(2 * (size_t)ni);
    for (int64_t chunk = 1; nrun < nsteps && build_err == QMC_OK; chunk *= 2) {
        const int64_t end = std::min(nsteps, nrun + chunk);
        wait_built(job0[end]);
        int64_t i = nrun;
        for (; i < end && build_err == QMC_OK; ++i) {
            for (int64_t j = job0[i]; j < job0[i + 1]; ++j) {
                int64_t off = 0;
                if ((build_err = add_prog(j, &off)) != QMC_OK) break;
                tab[2 * jobs[j].k + jobs[j].pass] = off;
                if (jobs[j].pass == 0) tab[2 * jobs[j].k + 1] = off;   // pass 1 repeats pass 0 when absent
                std::vector<uint8_t>().swap(built[j]);   // in the blob now (or shared with the step before)
            }
            if (build_err != QMC_OK) break;
            const size_t at = (blob.size() + 15) & ~(size_t)15;
            blob.resize(at + tab.size() * sizeof(int64_t));
            std::memcpy(blob.data() + at, tab.data(), tab.size() * sizeof(int64_t));
            info[i].tab_off = (int64_t)at;
        }
        const int64_t stop = i;   // steps [nrun, stop) are complete
        if (stop == nrun) break;
        if ((int64_t)blob.size() > std::min(ctx->progs_cap, ctx->h_progs_cap)) {
            // room for the whole call as the steps so far suggest
            const int64_t per = (int64_t)blob.size() / stop;
            const int64_t want = (int64_t)blob.size() + per * (nsteps - stop) * 5 / 4 + 65536;
            if (uploaded > 0) CK(cudaStreamSynchronize(ctx->work));   // the staging is rewritten below
            if ((rc = ensure_progs(ctx, want)) != QMC_OK) return rc;
            uploaded = 0;   // a new device buffer: copy every program again
        }
        const int64_t nb = (int64_t)blob.size() - uploaded;
        std::memcpy(ctx->h_progs + uploaded, blob.data() + uploaded, (size_t)nb);
        CK(cudaMemcpyAsync(ctx->d_progs + uploaded, ctx->h_progs + uploaded, (size_t)nb, cudaMemcpyHostToDevice,
                           ctx->work));
        uploaded = (int64_t)blob.size();
        std::memcpy(ctx->h_info + nrun, info.data() + nrun, (size_t)(stop - nrun) * sizeof(StepInfo));
        CK(cudaMemcpyAsync(ctx->d_info + nrun, ctx->h_info + nrun, (size_t)(stop - nrun) * sizeof(StepInfo),
                           cudaMemcpyHostToDevice, ctx->work));
        if ((rc = capture_graph(ctx)) != QMC_OK) return rc;
        for (int64_t s = nrun; s < stop; ++s) {
            if ((rc = note_launches(ctx, 1)) != QMC_OK) return rc;
            CK(cudaGraphLaunch(ctx->graph, ctx->work));
        }
        nrun = stop;
    }
    if (nrun == 0) {
        leave(ctx);
        return build_err;
    }
    int64_t done = 0;
    for (int attempt = 0; attempt < 64; ++attempt) {
        if (attempt > 0) {   // the first attempt's steps were launched above
            if ((rc = capture_graph(ctx)) != QMC_OK) return rc;
            for (int64_t i = done; i < nrun; ++i) {
                if ((rc = note_launches(ctx, 1)) != QMC_OK) return rc;
                CK(cudaGraphLaunch(ctx->graph, ctx->work));
            }
        }
        DevState hs;
        CK(cudaMemcpyAsync(&hs, ctx->d_state, sizeof(hs), cudaMemcpyDeviceToHost, ctx->work));
        CK(cudaStreamSynchronize(ctx->work));
        done = hs.call_index;
        if (!hs.error) break;
        const uint32_t code = hs.error;
        if ((rc = clear_dev_error(ctx)) != QMC_OK) return rc;
        if (ctx->wide) {
            // a failed wide step may have left merge scratch behind: zero it for the redo
            CK(cudaMemsetAsync(ctx->d_wdelta, 0, (size_t)(ctx->pop_cap + 1) * sizeof(int2), ctx->work));
            CK(cudaMemsetAsync(ctx->d_wnewcnt, 0, (size_t)(ctx->pop_cap + 1) * sizeof(int32_t), ctx->work));
            CK(cudaMemsetAsync(ctx->d_wmtile, 0, (size_t)ctx->wmtiles_cap * 8, ctx->work));
        }
        if (code == DERR_SPAWN_CAPACITY) {
            if ((rc = grow_spawn(ctx, hs.spawn_total)) != QMC_OK) return rc;
            if ((rc = grow_merge_tiles(ctx)) != QMC_OK) return rc;
        } else if (code == DERR_CAND_CAPACITY) {
            if ((rc = grow_cand(ctx, hs.cand_total)) != QMC_OK) return rc;
        } else if (code == DERR_HEAVY_CAPACITY) {
            const int64_t cap = std::max<int64_t>(hs.heavy_total * 2, ctx->heavy_cap * 2);
            if ((rc = dalloc(ctx, &ctx->d_heavy, cap)) != QMC_OK) return rc;
            ctx->heavy_cap = cap;
            ctx->graph_dirty = true;
        } else if (code == DERR_POP_CAPACITY) {
            if ((rc = grow_pop(ctx, hs.next_total)) != QMC_OK) return rc;
        } else if (code == DERR_TILE_CAPACITY) {
            if ((rc = grow_merge_tiles(ctx)) != QMC_OK) return rc;
            if ((rc = grow_spawn(ctx, ctx->spawn_cap)) != QMC_OK) return rc;
        } else {
            // fatal for this call: the state is that of the last completed step
            ctx->step += (uint64_t)done;
            if (done > 0) {
                ctx->t_prev = t0 + (double)(done - 1) * dt;
                ctx->t = t0 + (double)done * dt;
                ctx->dt_last = dt;
                ctx->prev_valid = true;
            }
            ctx->last_call_steps = done;
            leave(ctx);
            return map_dev_error(ctx, code, hs.error_aux);
        }
        // redo from the failed step
        ctx->acc_redo += nrun - done;
        CK(cudaMemcpyAsync((uint8_t*)ctx->d_state + offsetof(DevState, call_index), &done, 4,
                           cudaMemcpyHostToDevice, ctx->work));
        (void)zero;
    }
    if (done != nrun) return fail(ctx, QMC_ERR_CAPACITY, "could not complete the steps after growing buffers");
    ctx->step += (uint64_t)nrun;
    ctx->t_prev = t0 + (double)(nrun - 1) * dt;
    ctx->t = t0 + (double)nrun * dt;
    ctx->dt_last = dt;
    ctx->prev_valid = true;
    ctx->last_call_steps = nrun;
    // grow ahead of need so the next call rarely retries
    DevState hs;
    CK(cudaMemcpyAsync(&hs, ctx->d_state, sizeof(hs), cudaMemcpyDeviceToHost, ctx->work));
    CK(cudaStreamSynchronize(ctx->work));
    if (hs.max_spawn > ctx->spawn_cap * 3 / 4) {
        if ((rc = grow_spawn(ctx, hs.max_spawn * 2)) != QMC_OK) return rc;
        if ((rc = grow_merge_tiles(ctx)) != QMC_OK) return rc;
    }
    if (hs.max_cand > ctx->cand_cap * 3 / 4)
        if ((rc = grow_cand(ctx, hs.max_cand * 2)) != QMC_OK) return rc;
    if (hs.max_heavy > ctx->heavy_cap * 3 / 4) {
        const int64_t cap = hs.max_heavy * 2;
        if ((rc = dalloc(ctx, &ctx->d_heavy, cap)) != QMC_OK) return rc;
        ctx->heavy_cap = cap;
        ctx->graph_dirty = true;
    }
    if (hs.max_next > ctx->pop_cap * 3 / 4 && (ctx->cfg.max_records == 0 || ctx->pop_cap < ctx->cfg.max_records))
        if ((rc = grow_pop(ctx, hs.max_next * 2)) != QMC_OK) return rc;
    if ((rc = leave(ctx)) != QMC_OK) return rc;
    return build_err;   // QMC_OK unless a later step's program could not be built
}

int qmc_step_history(qmc_ctx* ctx, qmc_obs* obs, int64_t cap_steps, int64_t* count)
{
    if (!ctx || !obs || !count) return QMC_ERR_INVALID_ARG;
    const int64_t nsteps = std::min(cap_steps, ctx->last_call_steps);
    *count = nsteps;
    if (nsteps <= 0) return QMC_OK;
    int rc;
    if ((rc = enter(ctx)) != QMC_OK) return rc;
    std::vector<SegStats> h((size_t)nsteps * ctx->cfg.n_segments);
    CK(cudaMemcpyAsync(h.data(), ctx->d_history, h.size() * sizeof(SegStats), cudaMemcpyDeviceToHost, ctx->work));
    CK(cudaStreamSynchronize(ctx->work));
    for (size_t i = 0; i < h.size(); ++i)
        obs[i] = qmc_obs{(int64_t)h[i].count, h[i].ntot, h[i].dre, h[i].dim};
    return leave(ctx);
}

int qmc_z_history(qmc_ctx* ctx, int64_t* out, int64_t cap_steps, int64_t* count)
{
    if (!ctx || !out || !count) return QMC_ERR_INVALID_ARG;
    const int64_t nsteps = std::min(cap_steps, ctx->last_call_steps);
    *count = nsteps;
    if (nsteps <= 0) return QMC_OK;
    int rc;
    if ((rc = enter(ctx)) != QMC_OK) return rc;
    CK(cudaMemcpyAsync(out, ctx->d_zhist, (size_t)nsteps * ctx->cfg.n_segments * ctx->cfg.n_qubits * 8,
                       cudaMemcpyDeviceToHost, ctx->work));
    CK(cudaStreamSynchronize(ctx->work));
    return leave(ctx);
}

int qmc_export(qmc_ctx* ctx, int32_t seg, int32_t which, uint64_t* keys, int32_t* re, int32_t* im, int64_t cap,
               int64_t* count)
{
    if (!ctx || !count || seg < 0 || seg >= ctx->cfg.n_segments || (which != 0 && which != 1))
        return QMC_ERR_INVALID_ARG;
    if (ctx->wide) return fail(ctx, QMC_ERR_INVALID_ARG, "keys exceed 64 bits above 32 qubits: use qmc_export_xy");
    int rc;
    if ((rc = enter(ctx)) != QMC_OK) return rc;
    DevState hs;
    CK(cudaMemcpyAsync(&hs, ctx->d_state, sizeof(hs), cudaMemcpyDeviceToHost, ctx->work));
    CK(cudaStreamSynchronize(ctx->work));
    const int slot = which == 0 ? hs.cur : (hs.cur + 2) % 3;
    int64_t off[2];
    CK(cudaMemcpyAsync(off, ctx->d_segoff[slot] + seg, 16, cudaMemcpyDeviceToHost, ctx->work));
    CK(cudaStreamSynchronize(ctx->work));
    const int64_t cnt = off[1] - off[0];
    *count = cnt;
    if (cnt > cap) return fail(ctx, QMC_ERR_INVALID_ARG, "export capacity too small");
    if (cnt > 0) {
        std::vector<Rec> r(cnt);
        CK(cudaMemcpyAsync(r.data(), ctx->d_pop[slot] + off[0], cnt * sizeof(Rec), cudaMemcpyDeviceToHost, ctx->work));
        CK(cudaStreamSynchronize(ctx->work));
        for (int64_t i = 0; i < cnt; ++i) {
            keys[i] = r[i].key;
            re[i] = r[i].re;
            im[i] = r[i].im;
        }
    }
    return leave(ctx);
}

int qmc_export_xy(qmc_ctx* ctx, int32_t seg, int32_t which, uint64_t* x, uint64_t* y, int32_t* re, int32_t* im,
                  int64_t cap, int64_t* count)
{
    if (!ctx || !count || seg < 0 || seg >= ctx->cfg.n_segments || (which != 0 && which != 1))
        return QMC_ERR_INVALID_ARG;
    const int n = instance_of(ctx, seg).n;
    if (!ctx->wide) {
        std::vector<uint64_t> keys((size_t)std::max<int64_t>(cap, 1));
        const int rc = qmc_export(ctx, seg, which, keys.data(), re, im, cap, count);
        if (rc != QMC_OK) return rc;
        const uint64_t ymask = n == 64 ? ~0ull : ((1ull << n) - 1ull);
        for (int64_t i = 0; i < *count && i < cap; ++i) {
            x[i] = keys[i] >> n;
            y[i] = keys[i] & ymask;
        }
        return QMC_OK;
    }
    int rc;
    if ((rc = enter(ctx)) != QMC_OK) return rc;
    DevState hs;
    CK(cudaMemcpyAsync(&hs, ctx->d_state, sizeof(hs), cudaMemcpyDeviceToHost, ctx->work));
    CK(cudaStreamSynchronize(ctx->work));
    const int slot = which == 0 ? hs.cur : (hs.cur + 2) % 3;
    int64_t off[2];
    CK(cudaMemcpyAsync(off, ctx->d_segoff[slot] + seg, 16, cudaMemcpyDeviceToHost, ctx->work));
    CK(cudaStreamSynchronize(ctx->work));
    const int64_t cnt = off[1] - off[0];
    *count = cnt;
    if (cnt > cap) return fail(ctx, QMC_ERR_INVALID_ARG, "export capacity too small");
    if (cnt > 0) {
        uint64_t *d_x = nullptr, *d_y = nullptr;
        int32_t *d_re = nullptr, *d_im = nullptr;
        Scratch tmp(ctx);
        if ((rc = tmp.get(&d_x, cnt)) != QMC_OK || (rc = tmp.get(&d_y, cnt)) != QMC_OK ||
            (rc = tmp.get(&d_re, cnt)) != QMC_OK || (rc = tmp.get(&d_im, cnt)) != QMC_OK)
            return rc;
        launch_wide_export(params(ctx), slot, off[0], cnt, d_x, d_y, d_re, d_im, ctx->work);
        CK(cudaGetLastError());
        CK(cudaMemcpyAsync(x, d_x, cnt * 8, cudaMemcpyDeviceToHost, ctx->work));
        CK(cudaMemcpyAsync(y, d_y, cnt * 8, cudaMemcpyDeviceToHost, ctx->work));
        CK(cudaMemcpyAsync(re, d_re, cnt * 4, cudaMemcpyDeviceToHost, ctx->work));
        CK(cudaMemcpyAsync(im, d_im, cnt * 4, cudaMemcpyDeviceToHost, ctx->work));
        CK(cudaStreamSynchronize(ctx->work));
    }
    return leave(ctx);
}

} // extern "C"

// ---------------------------------------------------------------------------
// observables, overlap, checkpoint / restore
// ---------------------------------------------------------------------------
namespace {

struct CkptHeader {
    char magic[8];
    uint32_t version;
    int32_t n_qubits;
    uint64_t hash;
    uint64_t step;
    double t, t_prev, dt_last;
    int32_t prev_valid;
    int32_t nseg;
    int64_t count[2];
};

uint64_t fnv(uint64_t h, const void* p, size_t len)
{
    const uint8_t* b = (const uint8_t*)p;
    for (size_t i = 0; i < len; ++i) {
        h ^= b[i];
        h *= 1099511628211ull;
    }
    return h;
}

} // namespace

extern "C" {

int qmc_observables(qmc_ctx* ctx, qmc_obs* obs)
{
    if (!ctx || !obs) return QMC_ERR_INVALID_ARG;
    int rc;
    if ((rc = enter(ctx)) != QMC_OK) return rc;
    StepParams P = params(ctx);
    if (ctx->wide) {
        CK(cudaMemsetAsync(ctx->d_obs, 0, sizeof(SegStats) * (size_t)ctx->cfg.n_segments, ctx->work));
        launch_wide_obs(P, 0, ctx->d_obs, ctx->work);
    } else {
        launch_obs(P, 0, ctx->d_obs, ctx->grid, ctx->work);
    }
    CK(cudaGetLastError());
    std::vector<SegStats> h(ctx->cfg.n_segments);
    CK(cudaMemcpyAsync(h.data(), ctx->d_obs, h.size() * sizeof(SegStats), cudaMemcpyDeviceToHost, ctx->work));
    CK(cudaStreamSynchronize(ctx->work));
    for (size_t i = 0; i < h.size(); ++i) obs[i] = qmc_obs{(int64_t)h[i].count, h[i].ntot, h[i].dre, h[i].dim};
    return leave(ctx);
}

int qmc_overlap(qmc_ctx* ctx, int32_t seg, const uint64_t* idx, const double* psi_re, const double* psi_im,
                int32_t len, double* out_re, double* out_im)
{
    if (ctx && ctx->wide) return fail(ctx, QMC_ERR_INVALID_ARG, "qmc_overlap: not available above 32 qubits");
    if (!ctx || seg < 0 || seg >= ctx->cfg.n_segments || len < 0 || !out_re || !out_im) return QMC_ERR_INVALID_ARG;
    const int n = instance_of(ctx, seg).n;
    const int nq = len * len;
    std::vector<uint64_t> q(nq > 0 ? nq : 1);
    for (int a = 0; a < len; ++a)
        for (int b = 0; b < len; ++b) q[a * len + b] = (idx[a] << n) | idx[b];
    int rc;
    if ((rc = enter(ctx)) != QMC_OK) return rc;
    uint64_t* d_q = nullptr;
    int64_t* d_v = nullptr;
    Scratch tmp(ctx);
    if ((rc = tmp.get(&d_q, nq)) != QMC_OK || (rc = tmp.get(&d_v, 2 * (int64_t)nq)) != QMC_OK) return rc;
    std::vector<int64_t> v(2 * (size_t)(nq > 0 ? nq : 1));
    if (nq) {
        CK(cudaMemcpyAsync(d_q, q.data(), nq * 8, cudaMemcpyHostToDevice, ctx->work));
        launch_lookup(params(ctx), seg, d_q, nq, d_v, ctx->work);
        CK(cudaGetLastError());
        CK(cudaMemcpyAsync(v.data(), d_v, 2 * (size_t)nq * 8, cudaMemcpyDeviceToHost, ctx->work));
    }
    CK(cudaStreamSynchronize(ctx->work));
    // sum_{a,b} conj(psi_a) N_ab psi_b in a fixed order
    double sr = 0.0, si = 0.0;
    for (int a = 0; a < len; ++a) {
        for (int b = 0; b < len; ++b) {
            const double nr = (double)v[2 * (a * len + b)], ni = (double)v[2 * (a * len + b) + 1];
            const double car = psi_re[a], cai = -psi_im[a];
            const double pr = car * nr - cai * ni, pi = car * ni + cai * nr;
            sr += pr * psi_re[b] - pi * psi_im[b];
            si += pr * psi_im[b] + pi * psi_re[b];
        }
    }
    *out_re = sr;
    *out_im = si;
    return leave(ctx);
}

namespace {
int aux_reserve(qmc_ctx* ctx, int64_t bytes)
{
    if (bytes <= ctx->aux_cap) return QMC_OK;
    int rc = dalloc(ctx, &ctx->d_aux, bytes);
    if (rc == QMC_OK) ctx->aux_cap = bytes;
    return rc;
}
} // namespace

} // extern "C"

namespace {

// qmc_overlap_all above 32 qubits: the len^2 values N_ab of every vector by
// device lookups, summed on the host in qmc_overlap's order.
int overlap_all_wide(qmc_ctx* ctx, const uint64_t* idx, const double* psi_re, const double* psi_im, int32_t len,
                     double* out_re, double* out_im)
{
    const int nseg = ctx->cfg.n_segments;
    const int nq = len * len;
    std::vector<uint64_t> qx(nq), qy(nq);
    for (int a = 0; a < len; ++a)
        for (int b = 0; b < len; ++b) {
            qx[a * len + b] = idx[a];
            qy[a * len + b] = idx[b];
        }
    int rc;
    if ((rc = enter(ctx)) != QMC_OK) return rc;
    uint64_t *d_qx = nullptr, *d_qy = nullptr;
    int64_t* d_v = nullptr;
    Scratch tmp(ctx);
    if ((rc = tmp.get(&d_qx, nq)) != QMC_OK || (rc = tmp.get(&d_qy, nq)) != QMC_OK ||
        (rc = tmp.get(&d_v, 2 * (int64_t)nq * nseg)) != QMC_OK)
        return rc;
    CK(cudaMemcpyAsync(d_qx, qx.data(), 8 * (size_t)nq, cudaMemcpyHostToDevice, ctx->work));
    CK(cudaMemcpyAsync(d_qy, qy.data(), 8 * (size_t)nq, cudaMemcpyHostToDevice, ctx->work));
    const StepParams P = params(ctx);
    for (int s = 0; s < nseg; ++s) launch_wide_lookup(P, s, d_qx, d_qy, nq, d_v + 2 * (int64_t)nq * s, ctx->work);
    CK(cudaGetLastError());
    std::vector<int64_t> v(2 * (size_t)nq * nseg);
    CK(cudaMemcpyAsync(v.data(), d_v, v.size() * 8, cudaMemcpyDeviceToHost, ctx->work));
    CK(cudaStreamSynchronize(ctx->work));
    for (int s = 0; s < nseg; ++s) {
        const int64_t* w = v.data() + 2 * (size_t)nq * s;
        double sr = 0.0, si = 0.0;
        for (int a = 0; a < len; ++a) {
            for (int b = 0; b < len; ++b) {
                const double nr = (double)w[2 * (a * len + b)], ni = (double)w[2 * (a * len + b) + 1];
                const double car = psi_re[a], cai = -psi_im[a];
                const double pr = car * nr - cai * ni, pi = car * ni + cai * nr;
                sr += pr * psi_re[b] - pi * psi_im[b];
                si += pr * psi_im[b] + pi * psi_re[b];
            }
        }
        out_re[s] = sr;
        out_im[s] = si;
    }
    return leave(ctx);
}

} // namespace

extern "C" {

int qmc_overlap_all(qmc_ctx* ctx, const uint64_t* idx, const double* psi_re, const double* psi_im, int32_t len,
                    double* out_re, double* out_im)
{
    if (!ctx || len < 1 || len > kMaxOverlapLen || !idx || !psi_re || !psi_im || !out_re || !out_im)
        return QMC_ERR_INVALID_ARG;
    if (!ctx->has_pop) return fail(ctx, QMC_ERR_STATE, "no population");
    const int nseg = ctx->cfg.n_segments;
    int nmin = 64;
    for (const auto& I : ctx->inst) nmin = std::min(nmin, (int)I.n);
    for (int a = 0; a < len; ++a)
        if (nmin < 64 && (idx[a] >> nmin)) return fail(ctx, QMC_ERR_INVALID_ARG, "target index >= 2^n");
    int rc;
    if (ctx->wide) return overlap_all_wide(ctx, idx, psi_re, psi_im, len, out_re, out_im);
    if ((rc = enter(ctx)) != QMC_OK) return rc;
    const int64_t bytes = 8 * (int64_t)len + 16 * (int64_t)len + 16 * (int64_t)nseg;
    if ((rc = aux_reserve(ctx, bytes)) != QMC_OK) return rc;
    std::vector<double> psi(2 * (size_t)len);
    for (int a = 0; a < len; ++a) {
        psi[2 * a] = psi_re[a];
        psi[2 * a + 1] = psi_im[a];
    }
    uint64_t* d_idx = (uint64_t*)ctx->d_aux;
    double* d_psi = (double*)(ctx->d_aux + 8 * len);
    double* d_out = (double*)(ctx->d_aux + 24 * len);
    CK(cudaMemcpyAsync(d_idx, idx, 8 * (size_t)len, cudaMemcpyHostToDevice, ctx->work));
    CK(cudaMemcpyAsync(d_psi, psi.data(), 16 * (size_t)len, cudaMemcpyHostToDevice, ctx->work));
    launch_overlap_all(params(ctx), d_idx, d_psi, len, d_out, ctx->work);
    CK(cudaGetLastError());
    std::vector<double> h(2 * (size_t)nseg);
    CK(cudaMemcpyAsync(h.data(), d_out, 16 * (size_t)nseg, cudaMemcpyDeviceToHost, ctx->work));
    CK(cudaStreamSynchronize(ctx->work));
    for (int s = 0; s < nseg; ++s) {
        out_re[s] = h[2 * s];
        out_im[s] = h[2 * s + 1];
    }
    return leave(ctx);
}

int qmc_antihermiticity(qmc_ctx* ctx, uint64_t* out)
{
    if (ctx && ctx->wide) return fail(ctx, QMC_ERR_INVALID_ARG, "qmc_antihermiticity: not available above 32 qubits");
    if (!ctx || !out) return QMC_ERR_INVALID_ARG;
    if (!ctx->has_pop) return fail(ctx, QMC_ERR_STATE, "no population");
    const int nseg = ctx->cfg.n_segments;
    int rc;
    if ((rc = enter(ctx)) != QMC_OK) return rc;
    if ((rc = aux_reserve(ctx, 16 * (int64_t)nseg)) != QMC_OK) return rc;
    launch_antiherm(params(ctx), (unsigned long long*)ctx->d_aux, ctx->grid, ctx->work);
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(out, ctx->d_aux, 16 * (size_t)nseg, cudaMemcpyDeviceToHost, ctx->work));
    CK(cudaStreamSynchronize(ctx->work));
    return leave(ctx);
}

int qmc_antihermiticity_sum(qmc_ctx* ctx, const int32_t* vectors, int32_t count, uint64_t* out)
{
    if (ctx && ctx->wide) return fail(ctx, QMC_ERR_INVALID_ARG, "qmc_antihermiticity_sum: not available above 32 qubits");
    if (!ctx || !vectors || !out || count < 1 || count > 65535) return QMC_ERR_INVALID_ARG;
    if (!ctx->has_pop) return fail(ctx, QMC_ERR_STATE, "no population");
    const int nseg = ctx->cfg.n_segments;
    std::vector<int32_t> v(vectors, vectors + count), sorted = v;
    std::sort(sorted.begin(), sorted.end());
    for (int i = 0; i < count; ++i) {
        if (sorted[i] < 0 || sorted[i] >= nseg) return fail(ctx, QMC_ERR_INVALID_ARG, "vector index out of range");
        if (i && sorted[i] == sorted[i - 1]) return fail(ctx, QMC_ERR_INVALID_ARG, "a vector is listed twice");
        if (instance_of(ctx, sorted[i]).n != instance_of(ctx, sorted[0]).n)
            return fail(ctx, QMC_ERR_INVALID_ARG, "listed vectors differ in qubit count");
    }
    int rc;
    if ((rc = enter(ctx)) != QMC_OK) return rc;
    if ((rc = aux_reserve(ctx, 16 + 4 * (int64_t)count)) != QMC_OK) return rc;
    int32_t* d_segs = (int32_t*)(ctx->d_aux + 16);
    CK(cudaMemcpyAsync(d_segs, v.data(), 4 * (size_t)count, cudaMemcpyHostToDevice, ctx->work));
    launch_antiherm_sum(params(ctx), d_segs, count, (unsigned long long*)ctx->d_aux, ctx->grid, ctx->work);
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(out, ctx->d_aux, 16, cudaMemcpyDeviceToHost, ctx->work));
    CK(cudaStreamSynchronize(ctx->work));
    return leave(ctx);
}

int qmc_checkpoint(qmc_ctx* ctx, const char* path)
{
    if (ctx && ctx->wide) return fail(ctx, QMC_ERR_INVALID_ARG, "qmc_checkpoint: not available above 32 qubits");
    if (!ctx || !path) return QMC_ERR_INVALID_ARG;
    if (!ctx->has_pop) return fail(ctx, QMC_ERR_STATE, "nothing to checkpoint");
    int rc;
    if ((rc = enter(ctx)) != QMC_OK) return rc;
    DevState hs;
    CK(cudaMemcpyAsync(&hs, ctx->d_state, sizeof(hs), cudaMemcpyDeviceToHost, ctx->work));
    CK(cudaStreamSynchronize(ctx->work));
    const int nseg = ctx->cfg.n_segments;
    CkptHeader h;
    std::memset(&h, 0, sizeof(h));
    std::memcpy(h.magic, "QMCCKPT1", 8);
    h.version = 1;
    h.n_qubits = ctx->cfg.n_qubits;
    h.hash = context_hash(ctx);
    h.step = ctx->step;
    h.t = ctx->t;
    h.t_prev = ctx->t_prev;
    h.dt_last = ctx->dt_last;
    h.prev_valid = ctx->prev_valid ? 1 : 0;
    h.nseg = nseg;
    const int slots[2] = {hs.cur, (hs.cur + 2) % 3};
    std::vector<int64_t> off[2];
    std::vector<Rec> recs[2];
    for (int w = 0; w < 2; ++w) {
        off[w].resize(nseg + 1);
        CK(cudaMemcpyAsync(off[w].data(), ctx->d_segoff[slots[w]], (nseg + 1) * 8, cudaMemcpyDeviceToHost, ctx->work));
        CK(cudaStreamSynchronize(ctx->work));
        h.count[w] = (w == 1 && !ctx->prev_valid) ? 0 : hs.count[slots[w]];
        if (w == 1 && !ctx->prev_valid) std::fill(off[w].begin(), off[w].end(), 0);
        recs[w].resize(h.count[w]);
        if (h.count[w])
            CK(cudaMemcpyAsync(recs[w].data(), ctx->d_pop[slots[w]], h.count[w] * sizeof(Rec), cudaMemcpyDeviceToHost,
                               ctx->work));
    }
    CK(cudaStreamSynchronize(ctx->work));
    uint64_t sum = 1469598103934665603ull;
    sum = fnv(sum, &h, sizeof(h));
    FILE* f = std::fopen(path, "wb");
    if (!f) return fail(ctx, QMC_ERR_IO, std::string("cannot open ") + path);
    bool ok = std::fwrite(&h, sizeof(h), 1, f) == 1;
    for (int w = 0; w < 2 && ok; ++w) {
        ok = ok && std::fwrite(off[w].data(), 8, off[w].size(), f) == off[w].size();
        sum = fnv(sum, off[w].data(), off[w].size() * 8);
        if (h.count[w]) {
            ok = ok && std::fwrite(recs[w].data(), sizeof(Rec), recs[w].size(), f) == recs[w].size();
            sum = fnv(sum, recs[w].data(), recs[w].size() * sizeof(Rec));
        }
    }
    ok = ok && std::fwrite(&sum, 8, 1, f) == 1;
    ok = (std::fclose(f) == 0) && ok;
    if (!ok) return fail(ctx, QMC_ERR_IO, "checkpoint write failed");
    return leave(ctx);
}

int qmc_restore(qmc_ctx* ctx, const char* path)
{
    if (ctx && ctx->wide) return fail(ctx, QMC_ERR_INVALID_ARG, "qmc_restore: not available above 32 qubits");
    if (!ctx || !path) return QMC_ERR_INVALID_ARG;
    if (!has_schedules(ctx)) return fail(ctx, QMC_ERR_STATE, "load the same schedule before restoring");
    FILE* f = std::fopen(path, "rb");
    if (!f) return fail(ctx, QMC_ERR_IO, std::string("cannot open ") + path);
    CkptHeader h;
    const int nseg = ctx->cfg.n_segments;
    bool ok = std::fread(&h, sizeof(h), 1, f) == 1;
    if (!ok || std::memcmp(h.magic, "QMCCKPT1", 8) != 0 || h.version != 1) {
        std::fclose(f);
        return fail(ctx, QMC_ERR_CHECKPOINT, "not a checkpoint of this library");
    }
    const uint64_t hash = context_hash(ctx);
    if (h.hash != hash || h.nseg != nseg || h.n_qubits != ctx->cfg.n_qubits || h.count[0] < 0 || h.count[1] < 0 ||
        h.count[0] > ((int64_t)1 << 34) || h.count[1] > ((int64_t)1 << 34)) {
        std::fclose(f);
        return fail(ctx, QMC_ERR_CHECKPOINT, "checkpoint from another configuration or schedule");
    }
    uint64_t sum = fnv(1469598103934665603ull, &h, sizeof(h));
    std::vector<int64_t> off[2];
    std::vector<Rec> recs[2];
    for (int w = 0; w < 2 && ok; ++w) {
        off[w].resize(nseg + 1);
        ok = ok && std::fread(off[w].data(), 8, off[w].size(), f) == off[w].size();
        sum = fnv(sum, off[w].data(), off[w].size() * 8);
        recs[w].resize(h.count[w]);
        if (h.count[w]) {
            ok = ok && std::fread(recs[w].data(), sizeof(Rec), recs[w].size(), f) == recs[w].size();
            sum = fnv(sum, recs[w].data(), recs[w].size() * sizeof(Rec));
        }
    }
    uint64_t stored = 0;
    ok = ok && std::fread(&stored, 8, 1, f) == 1;
    std::fclose(f);
    if (!ok || stored != sum) return fail(ctx, QMC_ERR_CHECKPOINT, "checkpoint truncated or checksum mismatch");
    for (int w = 0; w < 2; ++w)
        if (off[w][0] != 0 || off[w][nseg] != h.count[w])
            return fail(ctx, QMC_ERR_CHECKPOINT, "inconsistent segment offsets");
    int rc;
    if ((rc = enter(ctx)) != QMC_OK) return rc;
    const int64_t need = std::max(h.count[0], h.count[1]);
    if (need > ctx->pop_cap && (rc = grow_pop(ctx, need)) != QMC_OK) return rc;
    DevState hs;
    std::memset(&hs, 0, sizeof(hs));
    CK(cudaMemcpyAsync(&hs, ctx->d_state, sizeof(hs), cudaMemcpyDeviceToHost, ctx->work));
    CK(cudaStreamSynchronize(ctx->work));
    hs.cur = 0;
    hs.count[0] = h.count[0];
    hs.count[1] = 0;
    hs.count[2] = h.count[1];
    hs.step = h.step;
    hs.error = 0;
    const int slots[2] = {0, 2};
    for (int w = 0; w < 2; ++w) {
        if (h.count[w])
            CK(cudaMemcpyAsync(ctx->d_pop[slots[w]], recs[w].data(), h.count[w] * sizeof(Rec), cudaMemcpyHostToDevice,
                               ctx->work));
        CK(cudaMemcpyAsync(ctx->d_segoff[slots[w]], off[w].data(), (nseg + 1) * 8, cudaMemcpyHostToDevice, ctx->work));
    }
    CK(cudaMemcpyAsync(ctx->d_state, &hs, sizeof(hs), cudaMemcpyHostToDevice, ctx->work));
    CK(cudaStreamSynchronize(ctx->work));
    ctx->step = h.step;
    ctx->t = h.t;
    ctx->t_prev = h.t_prev;
    ctx->dt_last = h.dt_last;
    ctx->prev_valid = h.prev_valid != 0;
    ctx->has_pop = true;
    return leave(ctx);
}

} // extern "C"

extern "C" {

int qmc_step_profile(qmc_ctx* ctx, double dt, int64_t nsteps, double* kernel_ms, int32_t cap, int32_t* n_kernels)
{
    if (!ctx || !kernel_ms || !n_kernels || cap < 0) return QMC_ERR_INVALID_ARG;
    if (!has_schedules(ctx) || !ctx->has_pop) return fail(ctx, QMC_ERR_STATE, "load a schedule and populations first");
    if (!(dt > 0.0) || nsteps < 1) return fail(ctx, QMC_ERR_INVALID_ARG, "dt must be > 0 and nsteps >= 1");
    const int nk = ctx->wide ? kNumWideGroups : kNumTimedKernels;
    *n_kernels = nk;
    for (int i = 0; i < cap && i < nk; ++i) kernel_ms[i] = 0.0;
    cudaEvent_t ev[kNumTimedKernels + kNumWideGroups + 1];
    for (int i = 0; i <= nk; ++i) CK(cudaEventCreate(&ev[i]));
    int rc = QMC_OK;
    for (int64_t s = 0; s < nsteps && rc == QMC_OK; ++s) {
        // one ordinary step first, so programs, capacities and the clock are handled as in qmc_step
        // (a step that needs buffers to grow is redone there); then time the same launch sequence
        rc = qmc_step(ctx, dt, 1);
        if (rc != QMC_OK) break;
        // replay the step just taken: restore the pre-step slot and clock on the device
        DevState hs;
        CK(cudaMemcpyAsync(&hs, ctx->d_state, sizeof(hs), cudaMemcpyDeviceToHost, ctx->work));
        CK(cudaStreamSynchronize(ctx->work));
        DevState back = hs;
        back.cur = (hs.cur + 2) % 3;
        back.step = hs.step - 1;
        back.call_index = 0;
        CK(cudaMemcpyAsync(ctx->d_state, &back, sizeof(back), cudaMemcpyHostToDevice, ctx->work));
        StepParams P = params(ctx);
        if ((rc = note_launches(ctx, 1)) != QMC_OK) break;
        if (ctx->wide)
            launch_wide_step(P, wparams(ctx), ctx->work, ev);
        else
            launch_step(P, ctx->grid, ctx->work, ev);
        CK(cudaGetLastError());
        CK(cudaStreamSynchronize(ctx->work));
        DevState after;
        CK(cudaMemcpyAsync(&after, ctx->d_state, sizeof(after), cudaMemcpyDeviceToHost, ctx->work));
        CK(cudaStreamSynchronize(ctx->work));
        if (after.error || after.cur != hs.cur || after.count[hs.cur] != hs.count[hs.cur]) {
            rc = fail(ctx, QMC_ERR_STATE, "profiled replay of a step did not reproduce it");
            break;
        }
        // the replay is a measurement, not a step: the cumulative counters keep
        // the values of the step it repeated
        const size_t acc0 = offsetof(DevState, acc_steps), acc1 = offsetof(DevState, acc_sort_lsd) + 8;
        CK(cudaMemcpyAsync((uint8_t*)ctx->d_state + acc0, (const uint8_t*)&hs + acc0, acc1 - acc0,
                           cudaMemcpyHostToDevice, ctx->work));
        CK(cudaStreamSynchronize(ctx->work));
        for (int i = 0; i < nk && i < cap; ++i) {
            float ms = 0.f;
            CK(cudaEventElapsedTime(&ms, ev[i], ev[i + 1]));
            kernel_ms[i] += ms;
        }
    }
    for (int i = 0; i <= nk; ++i) cudaEventDestroy(ev[i]);
    return rc;
}

int qmc_step_launches(const qmc_ctx* ctx, int32_t* launches)
{
    if (!ctx || !launches) return QMC_ERR_INVALID_ARG;
    qmc_ctx* c = const_cast<qmc_ctx*>(ctx);
    *launches = c->wide ? wide_step_launch_count(params(c), wparams(c)) : step_launch_count(params(c));
    return QMC_OK;
}

const char* qmc_kernel_name(int32_t i)
{
    if (i < 0 || i >= kNumTimedKernels) return "";
    return kKernelNames[i];
}

const char* qmc_step_kernel_name(const qmc_ctx* ctx, int32_t i)
{
    if (ctx && ctx->wide) return (i >= 0 && i < kNumWideGroups) ? kWideGroupNames[i] : "";
    return qmc_kernel_name(i);
}

} // extern "C"

extern "C" int qmc_counters(qmc_ctx* ctx, int32_t reset, int64_t* out)
{
    if (!ctx || !out) return QMC_ERR_INVALID_ARG;
    int rc;
    if ((rc = enter(ctx)) != QMC_OK) return rc;
    DevState hs;
    CK(cudaMemcpyAsync(&hs, ctx->d_state, sizeof(hs), cudaMemcpyDeviceToHost, ctx->work));
    CK(cudaStreamSynchronize(ctx->work));
    out[0] = hs.acc_steps;
    out[1] = hs.acc_walkers;
    out[2] = hs.acc_kcur;
    out[3] = hs.acc_kprev;
    out[4] = hs.acc_spawn;
    out[5] = hs.acc_knext;
    out[6] = hs.acc_heavy;
    out[7] = hs.acc_cand;
    out[8] = hs.acc_sort_bucket;
    out[9] = hs.acc_sort_lsd;
    out[10] = ctx->acc_redo;
    if (reset) {
        ctx->acc_redo = 0;
        int64_t z[10] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
        CK(cudaMemcpyAsync((uint8_t*)ctx->d_state + offsetof(DevState, acc_steps), z, sizeof(z),
                           cudaMemcpyHostToDevice, ctx->work));
        CK(cudaStreamSynchronize(ctx->work));
    }
    return leave(ctx);
}
