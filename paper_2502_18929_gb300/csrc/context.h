// Library-internal definition of the opaque qmc_ctx (include/qmc.h).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <unordered_map>
#include <vector>

#include "../../include/qmc.h"
#include "kernels.h"
#include "wide.h"
#include "qmc_types.h"
#include "term_compiler.h"

using qmc::DevState;
using qmc::HeavyItem;
using qmc::Rec;
using qmc::Schedule;
using qmc::SegStats;
using qmc::SpawnCand;
using qmc::SRec;
using qmc::StepInfo;

struct qmc_ctx {
    qmc_config cfg{};
    cudaStream_t user_stream = nullptr;
    cudaStream_t work = nullptr;
    cudaEvent_t ev = nullptr;
    cudaMemPool_t pool = nullptr;                   // stream-ordered device memory (no alloc callback)
    std::unordered_map<void*, size_t> blocks;       // device blocks held, with their sizes
    int64_t held_bytes = 0;
    int device = 0;
    int sm_count = 0;
    int grid = 0;
    int heavy_walkers = qmc::kHeavyWalkers;   // launch shapes (qmc_set_tuning)
    int bucket_records = 24;
    uint32_t spin_limit = qmc::kDefaultSpinLimit;   // qmc_set_spin_limit

    // Problem instances: one for a context made by qmc_create, several for
    // qmc_batch_create.  Instance i owns segments [seg0, seg0 + nvec).
    struct Instance {
        Schedule sched;
        bool has_sched = false;
        int32_t n = 0, nvec = 0, seg0 = 0;
        uint64_t seed = 0;
        int64_t n_diag = 0, init_min = 0;
    };
    std::vector<Instance> inst;
    bool batch = false;
    int proposal = 0;   // spawn choice rule (qmc_set_proposal)
    float* d_mlp = nullptr;          // learned proposal network
    uint8_t* d_mlp_tc = nullptr;     // the same network in the tensor-core layout (null if it does not fit)
    uint64_t* d_mlp_mask = nullptr;
    int32_t* d_mlp_idx = nullptr;
    int mlp_in = 0, mlp_hidden = 0, mlp_out = 0;
    uint8_t* d_learn_prog = nullptr;   // training: program at the current time
    int64_t learn_prog_cap = 0;
    float* d_learn_scratch = nullptr;  // training: per-event activations and gradients
    int64_t learn_scratch_cap = 0;
    double* d_learn_small = nullptr;   // training: [0] event count (int64), [1] weight sum, [2] loss
    uint8_t* d_learn_tc = nullptr;     // tensor-core training: bf16 weights and per-event rows, partial gradients
    int64_t learn_tc_cap = 0;
    float mlp_eps = 0.f;
    bool has_pop = false;
    qmc::SegInfo* d_seginfo = nullptr;
    qmc::InstInfo* d_inst = nullptr;

    DevState* d_state = nullptr;
    Rec* d_pop[3] = {nullptr, nullptr, nullptr};
    int64_t* d_segoff[3] = {nullptr, nullptr, nullptr};
    int64_t* d_gofs[3] = {nullptr, nullptr, nullptr};   // rank-group offsets (written by each step's prologue)
    int64_t pop_cap = 0;
    SRec* d_spawn = nullptr;
    SRec* d_spawn_alt = nullptr;
    int64_t spawn_cap = 0;
    SpawnCand* d_cand = nullptr;
    uint32_t* d_bucket = nullptr;
    unsigned long long* d_bscan_status = nullptr;
    uint32_t* d_big_list = nullptr;
    int64_t cand_cap = 0;
    HeavyItem* d_heavy = nullptr;
    int64_t heavy_cap = 0;
    uint2* d_kd = nullptr;
    unsigned int* d_sort_hist = nullptr;
    unsigned long long* d_sort_status = nullptr;
    int64_t sort_tiles_cap = 0;
    int64_t* d_bseg = nullptr;
    int64_t* d_tile_start = nullptr;
    qmc::MTileG* d_mtiles = nullptr;
    unsigned long long* d_merge_status = nullptr;
    int64_t launches_since_clear = 0;   // step launches since the look-back status arrays were cleared
    int64_t merge_tiles_cap = 0;
    SegStats* d_segacc = nullptr;
    SegStats* d_history = nullptr;
    int64_t history_cap = 0;
    long long* d_zacc = nullptr;     // [nseg][32] diagonal sums of the step being merged
    long long* d_zhist = nullptr;    // [history_cap][nseg][n] N^diag <Z_q> per step of the last call
    uint8_t* d_aux = nullptr;        // scratch of the on-demand observables (overlaps, anti-Hermiticity)
    int64_t aux_cap = 0;
    StepInfo* d_info = nullptr;
    int64_t info_cap = 0;
    uint8_t* d_progs = nullptr;
    int64_t progs_cap = 0;
    // pinned host staging of a qmc_step call's step table and programs: each
    // chunk of steps is copied from a region no later chunk rewrites
    qmc::StepInfo* h_info = nullptr;
    int64_t h_info_cap = 0;
    uint8_t* h_progs = nullptr;
    int64_t h_progs_cap = 0;
    SegStats* d_obs = nullptr;

    // host mirror of the clock
    uint64_t step = 0;
    double t = 0.0, t_prev = 0.0, dt_last = 0.0;
    bool prev_valid = false;
    int64_t last_call_steps = 0;
    int64_t acc_redo = 0;   // step launches repeated after a buffer grew (qmc_counters out[10])

    // 33..60 qubits: 128-bit keys; each d_pop slot holds pop_cap 16-byte keys
    // followed by pop_cap 8-byte values (24 bytes a record, structure of
    // arrays) and the step is the wide kernels' (wide.cu)
    bool wide = false;
    qmc::WSpawn* d_wspawn = nullptr;
    qmc::WSpawn* d_wspawn_alt = nullptr;
    qmc::WRun* d_wrun = nullptr;
    int32_t* d_wflag_u = nullptr;
    int64_t* d_wscan_u = nullptr;
    int2* d_wdelta = nullptr;
    int32_t* d_wnewcnt = nullptr;
    unsigned long long* d_wmtile = nullptr;
    longlong2* d_wmbase = nullptr;
    int64_t* d_wabound = nullptr;
    uint32_t* d_wwin = nullptr;
    uint32_t* d_wbig = nullptr;
    uint32_t* d_wnbig = nullptr;
    int64_t wmtiles_cap = 0;
    int64_t* d_wscan_a = nullptr;
    int64_t* d_wpart = nullptr;
    int64_t wpart_cap = 0;
    uint32_t* d_whist = nullptr;
    uint32_t* d_wtile = nullptr;
    int64_t wtiles_cap = 0;
    uint32_t* d_wplan = nullptr;

    cudaGraphExec_t graph = nullptr;
    bool graph_dirty = true;

    std::string err;
};
