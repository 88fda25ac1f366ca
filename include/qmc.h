/*
 * qmc.h -- C ABI of the GB300 (sm_103a) library for one step of real-time
 * population-dynamics quantum Monte Carlo for noisy circuits
 * (Shen & Lidar, arXiv:2502.18929).
 *
 * The library evolves many independent, signed-integer, sparse population
 * vectors N(t) over the vectorised density matrix |rho>> [walker averaging,
 * Eq. (3)] under the Liouvillian L(t) of the time-local master equation
 * [Eq. (1), Eq. (2)].  One step = spawning over L's Hamiltonian and Lindblad
 * terms (diagonal "death" included) [End Matter, spawn step], annihilation of
 * opposite signs on equal states [End Matter, annihilation step], the
 * initiator rule [End Matter, simulation methodology] and the per-vector
 * observables N^diag, N_tot, K [End Matter, sign-problem suppression].
 *
 * Conventions (all entry points):
 *   - Every call returns QMC_OK (0) or a negative QMC_ERR_* code;
 *     qmc_last_error() gives a one-line reason.  Calls are not thread-safe on
 *     one context.
 *   - Pointers marked "host" are caller-owned host memory, borrowed for the
 *     duration of the call only.  Pointers marked "device" are device memory
 *     on the context's GPU.  The library owns all memory it allocates; it
 *     takes it from qmc_config.alloc / free when given, else from a
 *     stream-ordered memory pool of the context.
 *   - Keys: qubit q is bit q of a basis index; rho_xy lives at the packed key
 *     (x << n) | y, n = number of qubits (1 <= n <= 60).  Up to 32 qubits a
 *     key is one uint64_t and the calls that take or return keys use it; from
 *     33 qubits on a key has 2n > 64 bits and a state is given as its bit
 *     strings x and y (qmc_init_populations, qmc_export_xy, qmc_overlap_all).
 *   - Pauli strings are bit-mask pairs (xm, zm): I (0,0), X (1,0), Z (0,1),
 *     Hermitian Y (1,1) per qubit.
 *   - Work is issued on the stream given in qmc_config.cuda_stream (0 = the
 *     legacy default stream).  Entry points that return data to the host
 *     synchronise that stream.
 */
#ifndef QMC_H
#define QMC_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- error codes -------------------------------------------------------- */
#define QMC_OK 0
#define QMC_ERR_INVALID_ARG (-1)    /* bad argument or inconsistent sizes       */
#define QMC_ERR_OOM (-2)            /* device or host allocation failed        */
#define QMC_ERR_CAPACITY (-3)       /* buffers full; grown and retried inside  */
                                    /* qmc_step, surfaced only past max_records */
#define QMC_ERR_DT_TOO_LARGE (-4)   /* a spawn probability p >= 1               */
#define QMC_ERR_POP_OVERFLOW (-5)   /* |re| or |im| of a state exceeds 2^31-1   */
#define QMC_ERR_DEVICE_TIMEOUT (-6) /* a bounded device wait expired            */
#define QMC_ERR_CUDA (-7)           /* a CUDA runtime call failed               */
#define QMC_ERR_STATE (-8)          /* call out of order (e.g. step before init)*/
#define QMC_ERR_COEF_RANGE (-9)     /* |coefficient * rate * dt| >= 2^10        */
#define QMC_ERR_IO (-10)            /* checkpoint file could not be read/written*/
#define QMC_ERR_CHECKPOINT (-11)    /* checkpoint corrupt or from another setup */

#define QMC_MAX_QUBITS 60

#define QMC_EULER 0
#define QMC_AB2 1

#define QMC_RATE_CONST 0 /* rate(t) = a                      */
#define QMC_RATE_COS 1   /* rate(t) = a * cos(b * t + c)     */

typedef struct qmc_ctx qmc_ctx;

/* Device allocator supplied by the caller (e.g. a framework's caching
 * allocator).  alloc returns bytes of device memory usable in stream order
 * on cuda_stream (the context's own work stream), or null when out of
 * memory; free returns such a block, in stream order on the same stream.
 * user is passed through unchanged. */
typedef void* (*qmc_alloc_fn)(uint64_t bytes, void* cuda_stream, void* user);
typedef void (*qmc_free_fn)(void* ptr, void* cuda_stream, void* user);

/* Run configuration.  n_segments independent population vectors ("samples",
 * Eq. (3)) share one problem; each draws its own counter-based random stream
 * keyed by (seed, step, segment, key, walker). */
typedef struct {
    int32_t n_qubits;      /* 1..QMC_MAX_QUBITS (above 32: 128-bit keys, exact
                              spawn choice only, no batch)                     */
    int32_t n_segments;    /* number of independent vectors, >= 1                */
    int32_t integrator;    /* QMC_EULER or QMC_AB2 (AB2 starts with one Euler)   */
    int32_t max_ctas;      /* cap on the CTAs of each persistent or grid-stride
                              kernel of a step (0: fill the GPU); lets a small
                              problem run many tiles per CTA                    */
    uint64_t seed;
    int64_t n_diag;        /* N^diag: walkers on the diagonal of N(0) = N^diag rho(0) */
    int64_t initiator_min; /* initiator threshold ceil(xi N^diag) in walkers; 0 = off */
    int64_t capacity_hint; /* initial records per population buffer (0 = auto)   */
    int64_t max_records;   /* hard cap for automatic growth (0 = no cap)         */
    void* cuda_stream;     /* cudaStream_t to issue work on                     */
    qmc_alloc_fn alloc;    /* device memory: null (with free null) = a pool of
                              the context's own, cudaMallocFromPoolAsync /
                              cudaFreeAsync in stream order on its work stream,
                              so growing a buffer never synchronises the device */
    qmc_free_fn free;      /* set together with alloc                           */
    void* alloc_user;      /* passed to alloc and free                          */
} qmc_config;

/* One term h * rate(t) * window(t) * P of H(t) [Eq. (1)]. */
typedef struct {
    double h;
    uint64_t xm, zm;
    int32_t rate_id;   /* index into the rate table                           */
    int32_t window_id; /* index into the window table, -1 = always on         */
} qmc_ham_term;

/* One Pauli component l_a * P_a of a Lindblad operator L_k = sum_a l_a P_a. */
typedef struct {
    double re, im;
    uint64_t xm, zm;
} qmc_pauli_coef;

/* A Lindblad operator with rate gamma_k(t) [Eq. (1)]; gamma may be negative
 * (non-Markovian).  Its components are coefs[first .. first + count). */
typedef struct {
    int32_t first, count;
    int32_t rate_id, window_id;
} qmc_lindblad;

typedef struct { int32_t kind; int32_t pad; double a, b, c; } qmc_rate;
typedef struct { double t0, t1; } qmc_window; /* active on [t0, t1) */

/* Per-vector observables, exact integer sums over N(t).
 * N^diag = n_diag_re + i n_diag_im; theta = atan2(im, re) [sign-problem
 * suppression]; Tr rho_j = n_diag_re / N^diag [replica aggregation]. */
typedef struct {
    int64_t n_records; /* K: occupied states, dim(H_QMC) of this vector        */
    int64_t n_walkers; /* N_tot = sum |re| + |im|                               */
    int64_t n_diag_re;
    int64_t n_diag_im;
} qmc_obs;

/* ---- lifecycle --------------------------------------------------------- */

/* Create a context on the current CUDA device.  *out is set only on success.
 * With n_qubits > 32 the context steps 128-bit keys (records of 24 bytes)
 * with the same method and random stream; of the calls below it supports
 * load_schedule, init_populations, step, observables, step_history,
 * counters, memory, export_xy and overlap_all, and the exact spawn choice
 * (the others return INVALID_ARG or STATE).
 * Errors: INVALID_ARG (n_qubits outside 1..QMC_MAX_QUBITS, n_segments < 1,
 * n_diag < 1), OOM, CUDA. */
int qmc_create(qmc_ctx** out, const qmc_config* cfg);

/* One problem instance of a batch: its own qubit count, population vectors,
 * seed, N^diag, initiator threshold and schedule (the arrays have the meaning
 * of qmc_load_schedule's; borrowed for the call only). */
typedef struct {
    int32_t n_qubits;       /* 1..32                                           */
    int32_t n_vectors;      /* >= 1                                            */
    uint64_t seed;
    int64_t n_diag;         /* >= 1                                            */
    int64_t initiator_min;  /* 0 = off                                         */
    const qmc_ham_term* ham;
    int32_t n_ham;
    int32_t n_lind;
    const qmc_lindblad* lind;
    const qmc_pauli_coef* coefs;
    int32_t n_coefs;
    int32_t n_rates;
    const qmc_rate* rates;
    const qmc_window* windows;
    int32_t n_windows;
    int32_t pad;
} qmc_instance;

/* Batched step (no counterpart in the paper; its vectors are independent by
 * Eq. (3), so independent problems can share every launch).  Create one
 * context for n_instances problem instances: instance i's vectors are the
 * segments [sum_{j<i} n_vectors_j, ... + n_vectors_i) of every per-vector
 * call (observables, export, overlap, history).  A vector draws exactly the
 * random numbers it would draw in a context of its instance alone made by
 * qmc_create with the same seed (its index inside the instance keys the
 * stream), so each instance's populations are bit-identical to such a run.
 * All instances share dt, the clock and integrator, capacity_hint,
 * max_records, max_ctas, cuda_stream and the allocator from cfg (cfg's n_qubits,
 * n_segments, seed, n_diag and initiator_min are ignored).
 * qmc_init_populations gives every instance the same rho(0) (its (x, y)
 * must fit the smallest instance); qmc_load_schedule is refused (STATE).
 * Errors: INVALID_ARG (an instance out of range, a schedule that does not
 * validate, more than 2^28 vectors), OOM, CUDA. */
int qmc_batch_create(qmc_ctx** out, const qmc_instance* inst, int32_t n_instances, const qmc_config* cfg);

/* Free all device and host memory of the context (NULL is a no-op). */
void qmc_destroy(qmc_ctx* ctx);

/* One-line description of the last error on this context (never NULL). */
const char* qmc_last_error(const qmc_ctx* ctx);

/* ---- problem ------------------------------------------------------------ */

/* Destination choice of the spawn step.
 * QMC_PROPOSAL_EXACT (default): the paper's rule [End Matter, spawn step] --
 *   a walker spawns with probability p = dt sum_kl (|Re L| + |Im L|) and
 *   picks (destination, channel) with probability |c(L)| / sum.
 * QMC_PROPOSAL_STATIC (no counterpart in the paper): a walker attempts with
 *   p_att = the sum over destinations of their static weights (each
 *   destination's sum of |Re| + |Im| over its expanded, quantised terms, a
 *   bound on |Re L| + |Im L| for every state), picks a destination with
 *   probability static weight / p_att, and spawns onto its Re or Im channel
 *   with probabilities |Re L| / static weight and |Im L| / static weight.
 *   Every destination and channel receives the same expected spawn as with
 *   the exact rule, and only the chosen destination's element is evaluated.
 * Applies from the next qmc_step.  Errors: INVALID_ARG. */
#define QMC_PROPOSAL_EXACT 0
#define QMC_PROPOSAL_STATIC 1
#define QMC_PROPOSAL_LEARNED 2
/* QMC_PROPOSAL_LEARNED_TC (no counterpart in the paper): the learned
 * proposal with its network evaluated on the tensor cores -- bf16 weights
 * and activations, fp32 accumulation (mma.sync m16n8k16), GELU (tanh form,
 * the hardware tanh approximation) in place of ReLU, exp by CUDA's
 * single-precision function -- 16 sources per
 * warp.  The walker law is unbiased for any proposal, so this mode draws
 * from the same expected spawns as the others; its integer weights Q follow
 * the same construction as QMC_PROPOSAL_LEARNED's but are not reproducible
 * bit for bit on a CPU.  Needs a network with 16, 32, 48 or 64 hidden units,
 * at most 256 outputs and 80 inputs (INVALID_ARG otherwise). */
#define QMC_PROPOSAL_LEARNED_TC 3
int qmc_set_proposal(qmc_ctx* ctx, int32_t kind);

/* Network of the learned proposal (no counterpart in the paper).  With
 * QMC_PROPOSAL_LEARNED the attempt is the static proposal's; the destination
 * is drawn from integer weights Q_k summing to 2^24 that mix the network's
 * softmax over the source's destinations (share 1 - eps) with the static
 * proposal (share eps, so every destination keeps Q_k >= 1), and each
 * channel receives floor(A) + Bernoulli(frac A) walkers with
 * A = |c(L)| 2^24 / (Q_k p_att): the same expected spawn as the exact rule.
 * Inputs: the n bits of x, the n bits of y (1.0 or 0.0) and t; two hidden
 * layers with ReLU; one logit per destination mask.  Single precision in a
 * fixed order (reproducible on the CPU), exp by a degree-7 polynomial of
 * 2^f.  At most 256 destinations per column (else qmc_step returns
 * INVALID_ARG).  Borrowed for the call (copied to the device). */
typedef struct {
    int32_t n_in;               /* 2 n_qubits + 1                          */
    int32_t n_hidden;           /* 1..64                                   */
    int32_t n_out;              /* 1..4096 destination masks               */
    float eps;                  /* static share, in (0, 1]                 */
    const uint64_t* out_masks;  /* n_out distinct masks (dx << n) | dy     */
    const float* w1;            /* n_hidden x n_in, row-major              */
    const float* b1;            /* n_hidden                                */
    const float* w2;            /* n_hidden x n_hidden                     */
    const float* b2;            /* n_hidden                                */
    const float* w3;            /* n_out x n_hidden                        */
    const float* b3;            /* n_out                                   */
} qmc_mlp;

/* Load the learned proposal's network (one context of one instance).
 * Errors: INVALID_ARG (sizes, masks not distinct), STATE (a batch), OOM. */
int qmc_set_proposal_mlp(qmc_ctx* ctx, const qmc_mlp* mlp);

/* ---- Training of the learned proposal (no counterpart in the paper) ----
 * The network is trained towards the heat-bath choice of the plain method
 * (destination share |Re L| + |Im L| over the column's sum) on events the
 * method generates.  Sizes come from the network loaded by
 * qmc_set_proposal_mlp; parameters are packed w1 [H x I], b1 [H],
 * w2 [H x H], b2 [H], w3 [G x H], b3 [G] (qmc_learn_param_count floats).
 * Every array argument is DEVICE memory owned by the caller; per-event
 * arrays are feature-major: element (row r, event e) at r * ld + e. */

/* Number of packed parameters.  Errors: STATE (no network). */
int qmc_learn_param_count(qmc_ctx* ctx, int64_t* n_params);

/* Training events from N(t) at the current time t: E = min(K, max_events)
 * parent records, record floor(e K / max_events) for event e (all K records
 * when K <= max_events), over the vectors' records in vector order.  Per
 * event: feat [2n + 1][max_events] (x bits, y bits as 1.0 / 0.0, then
 * float(t)); target [G][max_events]: for each output whose destination has a
 * positive static weight, float(double(w_k) / double(W)) with w_k = |Re| + |Im|
 * of the quantised column element of dt L(t) and W the sum over those
 * outputs (0 when W = 0), -1 for the other outputs; weight [max_events]:
 * float(|re| + |im|) of the parent, 0 when W = 0.  *n_events (host) = E.
 * Synchronises.  Errors: INVALID_ARG, STATE (no network, schedule or
 * populations), COEF_RANGE, OOM. */
int qmc_learn_events(qmc_ctx* ctx, double dt, int64_t max_events, float* feat, float* target, float* weight,
                     int64_t* n_events);

/* Weighted cross-entropy of the network's softmax over each event's present
 * outputs (target >= 0) against the targets, sum_e w_e CE_e / sum_e w_e, and
 * its gradient with respect to the packed parameters `params` (forward and
 * backward on the GPU in single precision, sums over events in a fixed
 * order).  grad: device, n_params floats; *loss (host) in double.
 * Synchronises.  Errors: INVALID_ARG (n_events outside [1, ld], events x
 * (4 H + G + 1) above 2^28), STATE, OOM. */
int qmc_learn_grad(qmc_ctx* ctx, const float* params, const float* feat, const float* target, const float* weight,
                   int64_t ld, int64_t n_events, float* grad, double* loss);

/* The learned proposal's integer weights Q_k (summing to 2^24) for count
 * sources |x[i]><y[i]| (host arrays, x, y < 2^n) under the static column of
 * dt_eff L(t), by the current proposal mode: QMC_PROPOSAL_LEARNED the FP32
 * network, the values the step uses bit for bit; QMC_PROPOSAL_LEARNED_TC the
 * tensor-core network as the step evaluates it.  Q[i * cap_slots + k] for
 * the column's static slot k (ascending destination mask; 0 where the slot
 * has width 0); *n_slots receives the slot count.  Errors: INVALID_ARG
 * (another mode, cap_slots too small, above 32 qubits), STATE (no schedule or
 * network), COEF_RANGE. */
int qmc_learned_weights(qmc_ctx* ctx, double t, double dt_eff, const uint64_t* x, const uint64_t* y, int32_t count,
                        int64_t* Q, int32_t cap_slots, int32_t* n_slots);

/* As qmc_learn_grad for the tensor-core proposal's network
 * (QMC_PROPOSAL_LEARNED_TC): inputs -> GELU -> GELU -> logits with the
 * weights and both hidden activations taken as bf16 and fp32 accumulation
 * (mma.sync m16n8k16), the same masked weighted cross-entropy; the
 * gradient flows through the bf16 roundings unchanged.  Weight gradients are
 * bf16 products over chunks of 4096 events, summed chunk by chunk in a fixed
 * order (deterministic).  Event arrays 16-byte aligned.  Errors: as
 * qmc_learn_grad, and INVALID_ARG when the network does not fit the tensor
 * cores (16, 32, 48 or 64 hidden units, at most 256 outputs, 80 inputs). */
int qmc_learn_grad_tc(qmc_ctx* ctx, const float* params, const float* feat, const float* target,
                      const float* weight, int64_t ld, int64_t n_events, float* grad, double* loss);

/* One Adam step (Kingma & Ba, 2015) on params with first and second moments
 * m, v (device, n_params floats each; zero before step t = 1).  Asynchronous
 * on the context's stream.  Errors: INVALID_ARG (count or hyperparameters). */
int qmc_learn_adam(qmc_ctx* ctx, float* params, const float* grad, float* m, float* v, int64_t n_params, int64_t t,
                   float lr, float beta1, float beta2, float eps);

/* Copy trained parameters (device, packed) into the network the learned
 * proposal evaluates.  Errors: STATE (no network). */
int qmc_learn_load(qmc_ctx* ctx, const float* params);

/* Load H(t) and the Lindblad operators [Eq. (1)].  The library expands
 * -i[H, rho] and gamma (L rho L^dag - 1/2 {L^dag L, rho}) into Pauli
 * superoperator terms and, per step, into the column tables of Eq. (2).
 * All arrays are host, copied.  Errors: INVALID_ARG (ids out of range, masks
 * beyond n qubits). */
int qmc_load_schedule(qmc_ctx* ctx,
                      const qmc_ham_term* ham, int32_t n_ham,
                      const qmc_lindblad* lind, int32_t n_lind,
                      const qmc_pauli_coef* coefs, int32_t n_coefs,
                      const qmc_rate* rates, int32_t n_rates,
                      const qmc_window* windows, int32_t n_windows);

/* N(0) := N^diag rho(0) for every vector [walker averaging, Eq. (3)]: each
 * entry rho_xy = re + i im (host arrays of length nnz, (x, y) distinct) is
 * scaled by N^diag and each component stochastically rounded (exact in the
 * mean).  Resets the clock to t = 0, step 0, no previous population.
 * Errors: INVALID_ARG (duplicate keys, x or y >= 2^n), POP_OVERFLOW, STATE
 * (no schedule loaded). */
int qmc_init_populations(qmc_ctx* ctx, const uint64_t* x, const uint64_t* y,
                         const double* re, const double* im, int64_t nnz);

/* Replace the population of every vector (which = 0: N(t), 1: N(t - dt)) with
 * host records (keys ascending within each vector; values nonzero).
 * counts[s] records for vector s, laid out back to back.  Used to start from
 * a given state.  Errors: INVALID_ARG (unsorted/duplicate keys), CAPACITY. */
int qmc_set_populations(qmc_ctx* ctx, int32_t which, const int64_t* counts,
                        const uint64_t* keys, const int32_t* re, const int32_t* im);

/* qmc_set_populations with states given as bit strings (any n): record i of
 * the concatenated host arrays is (re[i] + i im[i]) |x[i]><y[i]|, (x, y)
 * ascending within each vector.  Errors as qmc_set_populations. */
int qmc_set_populations_xy(qmc_ctx* ctx, int32_t which, const int64_t* counts, const uint64_t* x,
                           const uint64_t* y, const int32_t* re, const int32_t* im);

/* Set the clock: global step index (keys the random stream), t of N(t), and,
 * for AB2, the time and step size of the previous step.  prev_valid = 0 makes
 * the next step Euler. */
int qmc_set_clock(qmc_ctx* ctx, uint64_t step, double t, double t_prev, double dt_last,
                  int32_t prev_valid);
int qmc_get_clock(const qmc_ctx* ctx, uint64_t* step, double* t, double* t_prev,
                  double* dt_last, int32_t* prev_valid);

/* ---- the hot path --------------------------------------------------------- */

/* Advance every vector by nsteps steps of size dt.  Step i of the call uses
 * L(t0 + i dt), t0 = the clock at entry; AB2 steps also spawn from N(t - dt)
 * with L at the previous step's time [End Matter, simulation methodology].
 * Issued asynchronously on the context stream (captured once in a CUDA graph
 * and replayed); the column programs of the steps are built by host threads
 * while the device runs the steps already built; returns after checking the
 * device status word.  On CAPACITY the buffers grow and the failed step is
 * redone (the result is bit-identical: every draw is keyed by step, vector,
 * key and walker).  Errors: STATE, DT_TOO_LARGE, POP_OVERFLOW, CAPACITY (past
 * max_records), DEVICE_TIMEOUT, CUDA, COEF_RANGE or INVALID_ARG (a step's
 * column cannot be built: the steps before it complete), OOM.  After an
 * error the state is that of the last completed step. */
int qmc_step(qmc_ctx* ctx, double dt, int64_t nsteps);

/* Take nsteps steps like qmc_step (dt, nsteps >= 1), and time each kernel of
 * every step with CUDA events on the context's stream: each step is taken
 * once, then replayed kernel by kernel with events between the launches (the
 * replay reproduces the step exactly; a mismatch returns STATE).  Adds the
 * per-kernel milliseconds, summed over the steps, to host kernel_ms[0 .. cap)
 * (zeroed first) and sets *n_kernels; qmc_kernel_name(i) names kernel i.
 * The replays leave the cumulative counters (qmc_counters) as the steps set
 * them.  For measurement; slower than qmc_step (one synchronisation per step). */
int qmc_step_profile(qmc_ctx* ctx, double dt, int64_t nsteps, double* kernel_ms, int32_t cap,
                     int32_t* n_kernels);

/* Kernel launches of one step as the context would issue it now (host
 * *launches).  The count depends on n_qubits, n_segments and the current
 * spawn capacity (which picks the spawn sort); kernels that find no work for
 * a step still launch and are counted.  Errors: INVALID_ARG. */
int qmc_step_launches(const qmc_ctx* ctx, int32_t* launches);
const char* qmc_kernel_name(int32_t i);

/* Name of entry i of qmc_step_profile's output for this context (above 32
 * qubits the entries are groups of the wide step's kernels). */
const char* qmc_step_kernel_name(const qmc_ctx* ctx, int32_t i);

/* Launch shapes of the step (not in the paper; results never depend on
 * them: every draw is keyed by step, vector, key and walker, and the heavy
 * and light spawn paths produce the same spawns).
 *   max_ctas        CTAs of every persistent kernel (0: fill the GPU)
 *   heavy_walkers   parents with more walkers take the per-parent heavy path
 *                   (16 .. 2^20; default 256)
 *   bucket_records  target records per bucket of the spawn sort, which sets
 *                   the bucket digit's width (4 .. 256; default 24) */
typedef struct {
    int32_t max_ctas;
    int32_t heavy_walkers;
    int32_t bucket_records;
    int32_t pad;
} qmc_tuning;

/* Set or read the launch shapes.  Errors: INVALID_ARG (out of range). */
int qmc_set_tuning(qmc_ctx* ctx, const qmc_tuning* tuning);
int qmc_get_tuning(const qmc_ctx* ctx, qmc_tuning* tuning);

/* Autotuner: from the current state, time nsteps steps of size dt (1 .. 64)
 * under candidate launch shapes, one knob at a time (CTAs per kernel: the
 * whole GPU, two or one per SM; heavy threshold 64, 256, 1024 walkers;
 * bucket target 12, 24, 48 records), keep a candidate that is at least 2 %
 * faster, and leave the best shapes set.  The populations, clock and
 * counters are restored after every trial, so the state afterwards is the
 * state before (the steps after the call are bit-identical to those without
 * it).  *out (host, may be NULL) receives the chosen shapes.  Needs room for a
 * copy of N(t) and N(t - dt) on the device.  Errors: STATE, INVALID_ARG, OOM,
 * and any error of the steps themselves. */
int qmc_autotune(qmc_ctx* ctx, double dt, int32_t nsteps, qmc_tuning* out);

/* Upper bound of the spawn probability p over all states for a step of size
 * dt at time t (AB2 factor 3/2 included): sum over the expanded terms of
 * |Re c| + |Im c| times |rate| times dt.  Host-only; used to choose dt. */
int qmc_spawn_prob_bound(const qmc_ctx* ctx, double t, double dt, double* p_bound);

/* Bounded device waits.  A kernel that places its tile after other CTAs'
 * tiles (the decoupled look-back of the spawn sort, of the bucket scan and of
 * the merge [End Matter, annihilation step: the merged output's positions])
 * polls another CTA's status word at most `polls` times (about 64 ns apart
 * after the first 32) before it gives up: the step then returns
 * QMC_ERR_DEVICE_TIMEOUT with the wait's site and tile in qmc_last_error, the
 * context keeps the populations of the last completed step, and the next
 * qmc_step call (after the limit is raised again) repeats the failed step
 * bit-identically.  Default 2^22 polls; 0 makes every such wait fail at its
 * first poll (for tests of the failure path).  Waits on a CTA's own bulk
 * copies keep their fixed limit.  Errors: INVALID_ARG (above 2^30). */
int qmc_set_spin_limit(qmc_ctx* ctx, uint32_t polls);

/* Device memory the context holds (host out[2]): out[0] bytes, out[1]
 * blocks, whether from qmc_config.alloc or the context's pool. */
int qmc_memory(const qmc_ctx* ctx, int64_t* out);

/* ---- results --------------------------------------------------------------- */

/* Per-vector observables of N(t) into obs[0 .. n_segments) (host).
 * Synchronises the stream. */
int qmc_observables(qmc_ctx* ctx, qmc_obs* obs);

/* Records of one vector (which 0: N(t), 1: N(t - dt)) as bit strings, in key
 * order: record i is (re[i] + i im[i]) |x[i]><y[i]| (host arrays of cap
 * entries; *count receives the vector's record count, of which min(cap,
 * count) are written).  Any n.  Errors: INVALID_ARG. */
int qmc_export_xy(qmc_ctx* ctx, int32_t seg, int32_t which, uint64_t* x, uint64_t* y, int32_t* re, int32_t* im,
                  int64_t cap, int64_t* count);

/* Per-step observables of the last qmc_step call: host array of
 * nsteps * n_segments entries, step-major.  *count receives the number of
 * steps recorded (<= cap_steps). */
int qmc_step_history(qmc_ctx* ctx, qmc_obs* obs, int64_t cap_steps, int64_t* count);

/* Cumulative totals since the last reset, all vectors (host out[11]):
 * out[0] steps, [1] walker-steps (sum over steps of N_tot of N(t + dt)),
 * [2] records read from N(t), [3] records read from N(t - dt) (AB2 steps),
 * [4] spawn records, [5] records written to N(t + dt), [6] heavy work items,
 * [7] spawn candidates (walker draws below the step's bound on p, each
 * checked against the exact column), [8] steps whose spawn records were
 * sorted by buckets, [9] steps that took the LSD radix sort (a bucket too
 * large for the bucket sort), [10] step launches repeated because a buffer
 * had to grow first (a capacity error inside a qmc_step call: the steps from
 * the failed one on run again, bit-identically).  reset != 0 zeroes them
 * after reading.
 * Synchronises. */
int qmc_counters(qmc_ctx* ctx, int32_t reset, int64_t* out);

/* Copy the records of vector seg (which = 0: N(t), 1: N(t - dt)) to host
 * arrays of capacity cap; *count receives the number of records (if it
 * exceeds cap nothing is copied and INVALID_ARG is returned). */
int qmc_export(qmc_ctx* ctx, int32_t seg, int32_t which, uint64_t* keys, int32_t* re,
               int32_t* im, int64_t cap, int64_t* count);

/* Sum over the target support of conj(psi_x) psi_y N_xy for vector seg, as
 * exact integers accumulated in FP64 on the host (fidelity F = |value| /
 * N^diag for a normalised psi) [Markovian circuit dynamics].  psi given as
 * host arrays idx[len], (re, im)[len]. */
int qmc_overlap(qmc_ctx* ctx, int32_t seg, const uint64_t* idx, const double* psi_re,
                const double* psi_im, int32_t len, double* out_re, double* out_im);

/* N^diag <Z_q> of every vector after each step of the last qmc_step call
 * [walker averaging, Eq. (3): <Z_q> = Tr(Z_q rho), rho = N / N^diag]: host
 * out[step][vector][q] (q < n_qubits of the context) = sum over the diagonal
 * records of Re N_xx (-1)^(x_q), bit q of x being qubit q; entries with q at
 * or above a batch instance's own qubit count are 0.  Accumulated inside the
 * merge of each step.  *count receives the number of steps (<= cap_steps). */
int qmc_z_history(qmc_ctx* ctx, int64_t* out, int64_t cap_steps, int64_t* count);

/* Overlap of every vector of N(t) with a target |psi> on len <= 64 basis
 * states (host idx[len], psi_re[len], psi_im[len]; each idx < 2^n of every
 * instance): out_re/out_im[vector] = sum over a, b of conj(psi_a) N_ab psi_b,
 * evaluated on the device from the exact populations in the same order and
 * rounding as qmc_overlap (fidelity F = |value| / N^diag for a normalised
 * psi) [Markovian circuit dynamics].  One launch and one synchronisation for
 * all vectors.  Errors: INVALID_ARG, STATE (no population). */
int qmc_overlap_all(qmc_ctx* ctx, const uint64_t* idx, const double* psi_re, const double* psi_im, int32_t len,
                    double* out_re, double* out_im);

/* ||N - N^dagger||_F^2 of every vector of N(t), exactly, as host out[2 s]
 * (low 64 bits) and out[2 s + 1] (high 64 bits) [End Matter on Hermiticity
 * preservation: epsilon = ||rho - rho^dagger||_F, rho = N / N^diag, so
 * epsilon = sqrt(value) / N^diag for one vector].  Each record's transposed
 * state is found by binary search in its vector.  Synchronises. */
int qmc_antihermiticity(qmc_ctx* ctx, uint64_t* out);

/* ||S - S^dagger||_F^2 of the sum S of the listed vectors' N(t) (host
 * vectors[count], distinct, of equal qubit count), exactly, as host out[0]
 * (low 64 bits) and out[1] (high): the anti-Hermiticity of a replica
 * aggregate [End Matter on Hermiticity preservation; replica aggregation,
 * Markovian circuit dynamics: rho_QMC = S / N^diag_eff, so epsilon =
 * sqrt(value) / N^diag_eff].  Each record looks up its key and its transposed
 * key in every listed vector (binary search).  Errors: INVALID_ARG (count
 * outside 1..65535, an index out of range or repeated, mixed qubit counts),
 * STATE (no population).  Synchronises. */
int qmc_antihermiticity_sum(qmc_ctx* ctx, const int32_t* vectors, int32_t count, uint64_t* out);

/* ---- checkpoint / resume ------------------------------------------------- */

/* Write (clock, seed, configuration hash, N(t), N(t - dt)) to path; restore
 * reads it back into a context created with the same configuration and
 * schedule.  A resumed run is bit-identical to an uninterrupted one.
 * Errors: IO, CHECKPOINT (bad magic, checksum or configuration hash). */
int qmc_checkpoint(qmc_ctx* ctx, const char* path);
int qmc_restore(qmc_ctx* ctx, const char* path);

/* ---- observables without device allocation -------------------------------- */

/* Largest n_segments accepted by qmc_observables_noalloc. */
#define QMC_NOALLOC_MAX_SEGMENTS 4096

/* Per-vector observables (as qmc_observables) of a population the caller keeps
 * in device memory, computed without allocating any device memory.  The paper
 * has no counterpart; this entry point exists for callers that cannot call
 * cudaMalloc: code running under an external memory manager that has already
 * reserved the device memory, and code that must not risk the implicit
 * synchronisation cudaMalloc and cudaFree can cause.
 *   records      device, 16 bytes per record (uint64 key (x << n) | y,
 *                int32 re, int32 im), 16-byte aligned, sorted by vector
 *   seg_offsets  device, 8-byte aligned, n_segments + 1 nondecreasing int64
 *                offsets: vector s holds records [seg_offsets[s],
 *                seg_offsets[s + 1]) (empty vectors allowed; records before
 *                seg_offsets[0] are not read)
 *   out          device, n_segments qmc_obs, written
 *   cuda_stream  stream to issue the work on (0 = legacy default stream);
 *                the call returns without synchronising it.
 * The accumulators are a library-owned static device array of
 * QMC_NOALLOC_MAX_SEGMENTS entries (128 KiB), held by every GPU that loads the
 * library until the process exits.  The first call on a device looks up that
 * array's device address (set-up, once per device, with that device current);
 * make this first call before any stream capture.  Every call clears and
 * reuses the same array, so calls whose work overlaps on the GPU (other
 * streams, other threads) race: serialise them.
 * Errors: INVALID_ARG (null pointers, n_segments < 1 or above
 * QMC_NOALLOC_MAX_SEGMENTS, n_qubits outside 1..32, records not 16-byte
 * or seg_offsets not 8-byte aligned), CUDA (set-up or launch failed).
 * Each warp sums its records per vector in registers and adds the sums with
 * one set of atomics per vector it touches, so the cost is one read of the
 * records whatever the vector sizes. */
int qmc_observables_noalloc(const void* records, const int64_t* seg_offsets, int32_t n_segments,
                            int32_t n_qubits, qmc_obs* out, void* cuda_stream);

/* ---- host-only utility -------------------------------------------------- */

/* Compile the column of dt_eff * L(t) [Eq. (2)] exactly as qmc_step does and
 * evaluate it at the source state |x><y| on the host (no GPU needed): writes up
 * to cap destinations in the canonical (ascending mask) order -- mask =
 * (dx << n) | dy, value (vre + i vim) in units of 2^-52 -- and the spawn
 * weight P = 2^52 dt_eff sum (|Re L| + |Im L|) to *p_out [End Matter, spawn
 * step].  Schedule arrays as in qmc_load_schedule (host, borrowed).  Returns
 * the number of destinations, or INVALID_ARG / COEF_RANGE. */
int qmc_column_eval(int32_t n_qubits, const qmc_ham_term* ham, int32_t n_ham, const qmc_lindblad* lind,
                    int32_t n_lind, const qmc_pauli_coef* coefs, int32_t n_coefs, const qmc_rate* rates,
                    int32_t n_rates, const qmc_window* windows, int32_t n_windows, double t, double dt_eff,
                    uint64_t x, uint64_t y, int32_t cap, uint64_t* mask, uint64_t* mask_hi, int64_t* vre,
                    int64_t* vim, int64_t* p_out);

#ifdef __cplusplus
}
#endif

#endif /* QMC_H */
