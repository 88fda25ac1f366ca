/*
 * qmc_oracle.c -- CPU oracle for one step of real-time population-dynamics QMC
 * (Shen & Lidar, "Real-time sign-problem-suppressed QMC for noisy quantum
 * circuit simulations", arXiv:2502.18929).
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference legs of bench.py may load this file.  It shares no
 * code with the CUDA library: its Philox, Pauli algebra, Liouvillian column,
 * sampling and annihilation are written out here, plainly and slowly, one
 * parent and one walker at a time.  Build with -ffp-contract=off.
 *
 * What it computes (paper passages in brackets):
 *   - The Liouvillian column of an occupied state |x><y| [Eq. (1), Eq. (2)],
 *     evaluated term by term by applying Pauli strings to the ket and bra.
 *     Each expanded term's coefficient c * rate(t) * dt_eff is rounded to the
 *     grid 2^-52 ("quantised"), then the column's elements are exact integer
 *     sums of those (reading R1: exact integer weights, so the sum order does
 *     not matter).
 *   - Spawning [End Matter, spawn step]: N^sp ~ B(m, p) with
 *     p = dt * sum_kl (|Re L| + |Im L|), spread over (kl, channel) by a
 *     multinomial with probabilities |c(L)| / sum.  Written as m independent
 *     walkers, each with a uniform 52-bit draw T (see walker_T); the walker
 *     spawns iff T < P (P = p * 2^52) and then goes to the entry whose
 *     cumulative-weight interval holds T (reading R2).  The sign rule is the
 *     paper's: Re channel s * sgn(Re L), Im channel i * s * sgn(Im L).
 *   - Annihilation [End Matter, annihilation step]: spawned walkers are added
 *     to the current population key by key; opposite signs cancel; zeros go.
 *   - Initiator rule [End Matter, simulation methodology]: a spawn from a
 *     parent with fewer than xi N^diag walkers onto a state unoccupied in N(t)
 *     is discarded.  The threshold arrives as an integer walker count.
 *   - Euler and AB2 [End Matter, simulation methodology]: AB2 spawns from N(t)
 *     with dt_eff = 1.5 dt at L(t) and from N(t - dt) with dt_eff = 0.5 dt at
 *     L(t - dt), the latter with the opposite sign.  The first step (and the
 *     first after a change of dt) is Euler.
 *   - Initialisation N(0) = N^diag rho(0) [walker averaging, Eq. (3)]:
 *     stochastic rounding of each component.
 *   - Keys: the state |x><y| of n qubits (n <= 60) is the 2n-bit integer
 *     (x << n) | y, held in 128 bits; populations are sorted by it.
 *   - Proposal spawning (not in the paper; the library's optional
 *     alternative to the exact |L|-weighted choice): a walker attempts with
 *     p_att = the sum over destinations of their static weights (each
 *     destination's sum of |Re| + |Im| over its quantised terms, a bound on
 *     |Re L| + |Im L| for every state), picks a destination with probability
 *     static weight / p_att, and spawns onto its Re or Im channel with the
 *     exact element weights inside that interval: the expected spawn per
 *     destination and channel is the plain method's, without evaluating
 *     the rest of the column.
 *   - Learned proposal (not in the paper): the attempt is the same; the
 *     destination is drawn from integer weights Q_k (summing to 2^24) that mix
 *     a small network's softmax over the destinations with the static
 *     proposal (share eps), and each channel receives floor(A) +
 *     Bernoulli(frac A) walkers with A = w * 2^24 / (Q_k * p_att), so that the
 *     expectation is again w / 2^52 per walker.  The network runs in single
 *     precision with its operations in a fixed order (see mlp_logit), the
 *     exponential is the polynomial of mlp_exp, and A is one double-precision
 *     quotient, exactly as the library evaluates them.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_OK 0
#define ORC_ERR_INVALID_ARG (-1)
#define ORC_ERR_OOM (-2)
#define ORC_ERR_DT_TOO_LARGE (-4)
#define ORC_ERR_POP_OVERFLOW (-5)
#define ORC_ERR_STATE (-8)
#define ORC_ERR_COEF_RANGE (-9)

#define ONE_52 4503599627370496.0 /* 2^52 */
#define MAX_QUBITS 60

typedef unsigned __int128 okey;   /* (x << n) | y */
#define P_LIMIT (((int64_t)1) << 52)

/* ------------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as   */
/* easy as 1, 2, 3", SC'11): 10 rounds of the 4x32 round function with the   */
/* published multipliers and Weyl key increments.                           */
/* ------------------------------------------------------------------------ */
void orc_philox(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4])
{
    uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int round = 0; round < 10; ++round) {
        uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Stream layout (reading R3; the paper names no generator). */
#define TAG_STEP 0x53544550u /* per (step, segment) key derivation */
#define TAG_INIT 0x494E4954u /* per segment key for initial rounding */
#define KIND_INIT 1u
#define KIND_LEARNED 2u
#define KIND_GROUP 3u   /* walker 0 or 1 of four parents (one rank group) */
#define KIND_EXTRA 4u   /* further walkers of one parent, four per call */
#define KIND_LOW 5u     /* low 20 bits of one walker's draw */

static void derive_key(uint64_t seed, uint64_t step, uint32_t seg, uint32_t tag, uint32_t kd[2])
{
    uint32_t ctr[4] = {(uint32_t)step, (uint32_t)(step >> 32), seg, tag};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t out[4];
    orc_philox(ctr, key, out);
    kd[0] = out[0];
    kd[1] = out[1];
}

/* ------------------------------------------------------------------------ */
/* Problem description                                                     */
/* ------------------------------------------------------------------------ */
typedef struct { double h; uint64_t xm, zm; int rate, win; } ham_term;
typedef struct { double re, im; uint64_t xm, zm; } pauli_coef;
typedef struct { int start, count, rate, win; } lind_op;
typedef struct { int kind; double a, b, c; } rate_fn;
typedef struct { double t0, t1; } window_fn;

typedef struct {
    int n;
    int nh, nl, nr, nw;
    ham_term* ham;
    lind_op* lind;
    pauli_coef* lp;
    rate_fn* rates;
    window_fn* wins;
} problem;

void* orc_problem_new(int n,
                      int nh, const double* h, const uint64_t* hx, const uint64_t* hz,
                      const int32_t* hrate, const int32_t* hwin,
                      int nl, const int32_t* lstart, const int32_t* lcount,
                      const int32_t* lrate, const int32_t* lwin,
                      int nlp, const double* lre, const double* lim,
                      const uint64_t* lx, const uint64_t* lz,
                      int nr, const int32_t* rkind, const double* ra, const double* rb,
                      const double* rc,
                      int nw, const double* wt0, const double* wt1)
{
    if (n < 1 || n > MAX_QUBITS) return NULL;
    problem* p = (problem*)calloc(1, sizeof(problem));
    if (!p) return NULL;
    p->n = n; p->nh = nh; p->nl = nl; p->nr = nr; p->nw = nw;
    p->ham = (ham_term*)calloc((size_t)(nh > 0 ? nh : 1), sizeof(ham_term));
    p->lind = (lind_op*)calloc((size_t)(nl > 0 ? nl : 1), sizeof(lind_op));
    p->lp = (pauli_coef*)calloc((size_t)(nlp > 0 ? nlp : 1), sizeof(pauli_coef));
    p->rates = (rate_fn*)calloc((size_t)(nr > 0 ? nr : 1), sizeof(rate_fn));
    p->wins = (window_fn*)calloc((size_t)(nw > 0 ? nw : 1), sizeof(window_fn));
    for (int i = 0; i < nh; ++i) {
        p->ham[i].h = h[i]; p->ham[i].xm = hx[i]; p->ham[i].zm = hz[i];
        p->ham[i].rate = hrate[i]; p->ham[i].win = hwin[i];
    }
    for (int i = 0; i < nl; ++i) {
        p->lind[i].start = lstart[i]; p->lind[i].count = lcount[i];
        p->lind[i].rate = lrate[i]; p->lind[i].win = lwin[i];
    }
    for (int i = 0; i < nlp; ++i) {
        p->lp[i].re = lre[i]; p->lp[i].im = lim[i]; p->lp[i].xm = lx[i]; p->lp[i].zm = lz[i];
    }
    for (int i = 0; i < nr; ++i) {
        p->rates[i].kind = rkind[i]; p->rates[i].a = ra[i];
        p->rates[i].b = rb[i]; p->rates[i].c = rc[i];
    }
    for (int i = 0; i < nw; ++i) { p->wins[i].t0 = wt0[i]; p->wins[i].t1 = wt1[i]; }
    return p;
}

void orc_problem_free(void* pp)
{
    problem* p = (problem*)pp;
    if (!p) return;
    free(p->ham); free(p->lind); free(p->lp); free(p->rates); free(p->wins);
    free(p);
}

static double rate_value(const problem* p, int id, double t)
{
    const rate_fn* r = &p->rates[id];
    if (r->kind == 1) return r->a * cos(r->b * t + r->c);
    return r->a;
}

static int window_on(const problem* p, int id, double t)
{
    if (id < 0) return 1;
    return p->wins[id].t0 <= t && t < p->wins[id].t1;
}

/* ------------------------------------------------------------------------ */
/* Pauli strings on computational basis states.                            */
/* X|b> = |1-b>, Y|b> = i (-1)^b |1-b>, Z|b> = (-1)^b |b>.  A phase is i^k,  */
/* k in {0,1,2,3}.                                                          */
/* ------------------------------------------------------------------------ */
static void pauli_on_ket(int n, uint64_t xm, uint64_t zm, uint64_t x, uint64_t* x_out, int* k_out)
{
    int k = 0;
    for (int q = 0; q < n; ++q) {
        int xb = (int)((xm >> q) & 1u), zb = (int)((zm >> q) & 1u);
        int b = (int)((x >> q) & 1u);
        if (xb && zb) {              /* Y */
            k += 1 + (b ? 2 : 0);
            x ^= ((uint64_t)1) << q;
        } else if (xb) {             /* X */
            x ^= ((uint64_t)1) << q;
        } else if (zb) {             /* Z */
            k += b ? 2 : 0;
        }
    }
    *x_out = x;
    *k_out = k & 3;
}

typedef struct { int64_t re, im; } cint;

/* (a + ib) * i^k, exact */
static cint times_ik(cint z, int k)
{
    cint r;
    switch (k & 3) {
    case 0: r = z; break;
    case 1: r.re = -z.im; r.im = z.re; break;
    case 2: r.re = -z.re; r.im = -z.im; break;
    default: r.re = z.im; r.im = -z.re; break;
    }
    return r;
}

/* Round a coefficient to the grid 2^-52 (nearest, ties to even). */
static int quantise(double re, double im, cint* out)
{
    double a = re * ONE_52, b = im * ONE_52;
    if (!(fabs(a) < 4611686018427387904.0) || !(fabs(b) < 4611686018427387904.0))
        return ORC_ERR_COEF_RANGE; /* |c| >= 2^10: no such step can have p < 1 */
    out->re = (int64_t)nearbyint(a);
    out->im = (int64_t)nearbyint(b);
    return ORC_OK;
}

/* Column entries of dt_eff * L(t) for the source |x><y|: a small list of     */
/* destinations keyed by mask = (dx << n) | dy, kept sorted by that key.      */
typedef struct { okey mask; cint v; } col_entry;
typedef struct { col_entry* e; int len, cap; } column;

static int column_add(column* c, okey mask, cint v)
{
    int lo = 0, hi = c->len;
    while (lo < hi) {
        int mid = (lo + hi) / 2;
        if (c->e[mid].mask < mask) lo = mid + 1; else hi = mid;
    }
    if (lo < c->len && c->e[lo].mask == mask) {
        c->e[lo].v.re += v.re;
        c->e[lo].v.im += v.im;
        return ORC_OK;
    }
    if (c->len == c->cap) {
        int ncap = c->cap ? 2 * c->cap : 64;
        col_entry* ne = (col_entry*)realloc(c->e, (size_t)ncap * sizeof(col_entry));
        if (!ne) return ORC_ERR_OOM;
        c->e = ne;
        c->cap = ncap;
    }
    memmove(&c->e[lo + 1], &c->e[lo], (size_t)(c->len - lo) * sizeof(col_entry));
    c->e[lo].mask = mask;
    c->e[lo].v = v;
    c->len++;
    return ORC_OK;
}

/*
 * Column of dt_eff * L(t) at source |x><y| [Eq. (1), Eq. (2)].
 * Expanded terms (each quantised on its own, reading R1):
 *   -i[H, rho]:  for h P with s = rate(t) * dt_eff and v = h * s:
 *                (-i v) P rho      and   (+i v) rho P
 *   gamma(t) (L rho L^dag - 1/2 L^dag L rho - 1/2 rho L^dag L), L = sum_a l_a P_a,
 *                with s = gamma(t) * dt_eff, for every ordered pair (a, b):
 *                z = l_a conj(l_b) = (la.re lb.re + la.im lb.im, la.im lb.re - la.re lb.im)
 *                (s z) P_a rho P_b
 *                (-s/2) conj(z) P_a P_b rho    and   (-s/2) conj(z) rho P_a P_b
 * A bra-side string acts as <y|P = conj(phase of P|y>) <y'| (P Hermitian);
 * <y| P_a P_b is the conjugate of P_b P_a |y>.
 */
static int build_column(const problem* p, uint64_t x, uint64_t y, double t, double dt_eff,
                        column* col)
{
    const int n = p->n;
    col->len = 0;
    int rc;
    for (int i = 0; i < p->nh; ++i) {
        const ham_term* ht = &p->ham[i];
        if (!window_on(p, ht->win, t)) continue;
        double s = rate_value(p, ht->rate, t) * dt_eff;
        double v = ht->h * s;
        cint qk, qb;
        if ((rc = quantise(0.0, -v, &qk)) != ORC_OK) return rc;
        if ((rc = quantise(0.0, v, &qb)) != ORC_OK) return rc;
        uint64_t x2, y2;
        int kx, ky;
        pauli_on_ket(n, ht->xm, ht->zm, x, &x2, &kx);
        if ((rc = column_add(col, (okey)(x ^ x2) << n, times_ik(qk, kx))) != ORC_OK) return rc;
        pauli_on_ket(n, ht->xm, ht->zm, y, &y2, &ky);
        if ((rc = column_add(col, (okey)(y ^ y2), times_ik(qb, 4 - ky))) != ORC_OK) return rc;
    }
    for (int i = 0; i < p->nl; ++i) {
        const lind_op* lo = &p->lind[i];
        if (!window_on(p, lo->win, t)) continue;
        double s = rate_value(p, lo->rate, t) * dt_eff;
        double hs = -0.5 * s;
        for (int a = 0; a < lo->count; ++a) {
            const pauli_coef* la = &p->lp[lo->start + a];
            for (int b = 0; b < lo->count; ++b) {
                const pauli_coef* lb = &p->lp[lo->start + b];
                double zre = la->re * lb->re + la->im * lb->im;
                double zim = la->im * lb->re - la->re * lb->im;
                cint qj, qa;
                if ((rc = quantise(s * zre, s * zim, &qj)) != ORC_OK) return rc;
                if ((rc = quantise(hs * zre, -(hs * zim), &qa)) != ORC_OK) return rc;
                uint64_t xa, yb, u1, u2, v1, v2;
                int ka, kb, k1, k2, j1, j2;
                /* jump: P_a |x><y| P_b */
                pauli_on_ket(n, la->xm, la->zm, x, &xa, &ka);
                pauli_on_ket(n, lb->xm, lb->zm, y, &yb, &kb);
                if ((rc = column_add(col, ((okey)(x ^ xa) << n) | (y ^ yb),
                                     times_ik(qj, ka + 4 - kb))) != ORC_OK) return rc;
                /* ket side: P_a P_b |x> */
                pauli_on_ket(n, lb->xm, lb->zm, x, &u1, &k1);
                pauli_on_ket(n, la->xm, la->zm, u1, &u2, &k2);
                if ((rc = column_add(col, (okey)(x ^ u2) << n, times_ik(qa, k1 + k2))) != ORC_OK)
                    return rc;
                /* bra side: <y| P_a P_b = conj(P_b P_a |y>) */
                pauli_on_ket(n, la->xm, la->zm, y, &v1, &j1);
                pauli_on_ket(n, lb->xm, lb->zm, v1, &v2, &j2);
                if ((rc = column_add(col, (okey)(y ^ v2), times_ik(qa, 8 - j1 - j2))) != ORC_OK)
                    return rc;
            }
        }
    }
    return ORC_OK;
}

/* Static weight of every destination of dt_eff * L(t): the sum over its
 * expanded terms of |Re c| + |Im c| of the quantised coefficient (the Pauli
 * phases only permute and negate components, so this bounds |Re L| + |Im L|
 * of that destination for every source state).  Destination masks do not
 * depend on the state (a Pauli string flips the bits of its X part). */
static int build_static(const problem* p, double t, double dt_eff, column* col)
{
    const int n = p->n;
    col->len = 0;
    int rc;
    for (int i = 0; i < p->nh; ++i) {
        const ham_term* ht = &p->ham[i];
        if (!window_on(p, ht->win, t)) continue;
        double s = rate_value(p, ht->rate, t) * dt_eff;
        double v = ht->h * s;
        cint qk, qb;
        if ((rc = quantise(0.0, -v, &qk)) != ORC_OK) return rc;
        if ((rc = quantise(0.0, v, &qb)) != ORC_OK) return rc;
        cint a = {llabs(qk.re) + llabs(qk.im), 0}, b = {llabs(qb.re) + llabs(qb.im), 0};
        if ((rc = column_add(col, (okey)ht->xm << n, a)) != ORC_OK) return rc;
        if ((rc = column_add(col, (okey)ht->xm, b)) != ORC_OK) return rc;
    }
    for (int i = 0; i < p->nl; ++i) {
        const lind_op* lo = &p->lind[i];
        if (!window_on(p, lo->win, t)) continue;
        double s = rate_value(p, lo->rate, t) * dt_eff;
        double hs = -0.5 * s;
        for (int a = 0; a < lo->count; ++a) {
            const pauli_coef* la = &p->lp[lo->start + a];
            for (int b = 0; b < lo->count; ++b) {
                const pauli_coef* lb = &p->lp[lo->start + b];
                double zre = la->re * lb->re + la->im * lb->im;
                double zim = la->im * lb->re - la->re * lb->im;
                cint qj, qa;
                if ((rc = quantise(s * zre, s * zim, &qj)) != ORC_OK) return rc;
                if ((rc = quantise(hs * zre, -(hs * zim), &qa)) != ORC_OK) return rc;
                cint aj = {llabs(qj.re) + llabs(qj.im), 0}, aa = {llabs(qa.re) + llabs(qa.im), 0};
                if ((rc = column_add(col, ((okey)la->xm << n) | lb->xm, aj)) != ORC_OK) return rc;
                if ((rc = column_add(col, (okey)(la->xm ^ lb->xm) << n, aa)) != ORC_OK) return rc;
                if ((rc = column_add(col, (okey)(la->xm ^ lb->xm), aa)) != ORC_OK) return rc;
            }
        }
    }
    return ORC_OK;
}

/* Exported for tests: the quantised column, sorted by mask (low 64 bits in
 * mask, high 64 in mask_hi unless null).  Returns the number of entries
 * (which may exceed cap; only cap are written) or < 0. */
int orc_column(const void* pp, uint64_t x, uint64_t y, double t, double dt_eff, int cap,
               uint64_t* mask, uint64_t* mask_hi, int64_t* qre, int64_t* qim)
{
    const problem* p = (const problem*)pp;
    column col = {0, 0, 0};
    int rc = build_column(p, x, y, t, dt_eff, &col);
    if (rc != ORC_OK) { free(col.e); return rc; }
    for (int i = 0; i < col.len && i < cap; ++i) {
        mask[i] = (uint64_t)col.e[i].mask;
        if (mask_hi) mask_hi[i] = (uint64_t)(col.e[i].mask >> 64);
        qre[i] = col.e[i].v.re;
        qim[i] = col.e[i].v.im;
    }
    int len = col.len;
    free(col.e);
    return len;
}

/* Exported for tests: the static weights (see build_static), sorted by
 * mask.  Returns the number of entries (only cap are written) or < 0. */
int orc_static(const void* pp, double t, double dt_eff, int cap, uint64_t* mask, uint64_t* mask_hi,
               int64_t* weight)
{
    const problem* p = (const problem*)pp;
    column col = {0, 0, 0};
    int rc = build_static(p, t, dt_eff, &col);
    if (rc != ORC_OK) { free(col.e); return rc; }
    for (int i = 0; i < col.len && i < cap; ++i) {
        mask[i] = (uint64_t)col.e[i].mask;
        if (mask_hi) mask_hi[i] = (uint64_t)(col.e[i].mask >> 64);
        weight[i] = col.e[i].v.re;
    }
    int len = col.len;
    free(col.e);
    return len;
}

/* ------------------------------------------------------------------------ */
/* Populations                                                             */
/* ------------------------------------------------------------------------ */
typedef struct { okey key; int32_t re, im; } rec;
typedef struct { rec* r; int64_t len, cap; } pop;

typedef struct { okey key; int64_t re, im; int noninit; } spawn_rec;
typedef struct { spawn_rec* s; int64_t len, cap; } spawn_list;

typedef struct {
    const problem* prob;
    int nseg;
    uint64_t seed;
    int integrator;       /* 0 = Euler, 1 = AB2 */
    int64_t init_min;     /* initiator threshold in walkers (ceil(xi N^diag)); 0 = off */
    int64_t n_diag;
    unsigned char* active; /* segments stepped by orc_step (all by default) */
    pop* cur;
    pop* prev;
    uint64_t step;        /* global step index */
    double t, t_prev, dt_last;
    int prev_valid;
    int proposal;         /* 0: exact |L|-weighted choice; 1: static proposal; 2: learned */
    /* learned proposal: network (see mlp_logit) */
    int mlp_in, mlp_hidden, mlp_out;
    float* w1; float* b1; float* w2; float* b2; float* w3; float* b3;
    uint64_t* out_mask;   /* destination mask of each output, as given */
    float eps;            /* static share of the mixture */
} state;

/* ------------------------------------------------------------------------ */
/* Learned proposal arithmetic, single precision in a fixed order.          */
/* ------------------------------------------------------------------------ */
/* e^x for x <= 0: 2^(x log2 e) = 2^k 2^f, 2^f by its Taylor polynomial of
 * degree 7 in Horner form (fused multiply-adds), 2^k by the exponent bits. */
static float mlp_exp(float x)
{
    if (x < -87.0f) return 0.0f;
    const float y = x * 1.44269504f;
    const float k = floorf(y);
    const float f = y - k;
    float p = 1.52527338e-5f;
    p = fmaf(p, f, 1.54035304e-4f);
    p = fmaf(p, f, 1.33335581e-3f);
    p = fmaf(p, f, 9.61812911e-3f);
    p = fmaf(p, f, 5.55041087e-2f);
    p = fmaf(p, f, 2.40226507e-1f);
    p = fmaf(p, f, 6.93147181e-1f);
    p = fmaf(p, f, 1.0f);
    const uint32_t bits = (uint32_t)((int)k + 127) << 23;
    float scale;
    memcpy(&scale, &bits, 4);
    return p * scale;
}

/* Hidden layers for the source |x><y| at time t: inputs are the n bits of x,
 * the n bits of y (1 or 0) and t; ReLU after each layer.  h2 receives the
 * second hidden layer. */
static void mlp_hidden(const state* s, uint64_t x, uint64_t y, double t, float* h1, float* h2)
{
    const int n = s->prob->n, H = s->mlp_hidden, I = s->mlp_in;
    const float tf = (float)t;
    for (int j = 0; j < H; ++j) {
        float a = s->b1[j];
        for (int i = 0; i < 2 * n; ++i) {
            const uint64_t bit = i < n ? (x >> i) & 1u : (y >> (i - n)) & 1u;
            if (bit) a = a + s->w1[j * I + i];
        }
        a = fmaf(s->w1[j * I + 2 * n], tf, a);
        h1[j] = a > 0.0f ? a : 0.0f;
    }
    for (int j = 0; j < H; ++j) {
        float a = s->b2[j];
        for (int i = 0; i < H; ++i) a = fmaf(s->w2[j * H + i], h1[i], a);
        h2[j] = a > 0.0f ? a : 0.0f;
    }
}

static float mlp_logit(const state* s, const float* h2, int g)
{
    const int H = s->mlp_hidden;
    float a = s->b3[g];
    for (int i = 0; i < H; ++i) a = fmaf(s->w3[g * H + i], h2[i], a);
    return a;
}

/* Output index of a destination mask, or -1. */
static int mlp_output(const state* s, okey mask)
{
    for (int g = 0; g < s->mlp_out; ++g)
        if ((okey)s->out_mask[g] == mask) return g;
    return -1;
}

/* Integer proposal weights Q[0 .. st->len) (sum 2^24) of the source. */
static void learned_weights(const state* s, const column* st, int64_t p_att, uint64_t x, uint64_t y, double t,
                            int64_t* Q)
{
    float h1[64], h2[64];
    mlp_hidden(s, x, y, t, h1, h2);
    const int ns = st->len;
    float m = -INFINITY;
    for (int k = 0; k < ns; ++k) {
        const int g = st->e[k].v.re > 0 ? mlp_output(s, st->e[k].mask) : -1;
        if (g >= 0) {
            const float l = mlp_logit(s, h2, g);
            if (l > m) m = l;
        }
    }
    float S = 0.0f;
    for (int k = 0; k < ns; ++k) {
        const int g = st->e[k].v.re > 0 ? mlp_output(s, st->e[k].mask) : -1;
        if (g >= 0) S = S + mlp_exp(mlp_logit(s, h2, g) - m);
    }
    const float omeps = 1.0f - s->eps;
    int64_t sum = 0;
    int arg = -1;
    for (int k = 0; k < ns; ++k) {
        Q[k] = 0;
        if (st->e[k].v.re <= 0) continue;
        const int g = mlp_output(s, st->e[k].mask);
        int64_t L = 0;
        if (g >= 0 && S > 0.0f) {
            const float q = mlp_exp(mlp_logit(s, h2, g) - m) / S;
            L = (int64_t)floorf((omeps * q) * 16777216.0f);
        }
        const int64_t St = (int64_t)floor((double)s->eps * (double)st->e[k].v.re / (double)p_att * 16777216.0);
        Q[k] = L + St;
        if (Q[k] < 1) Q[k] = 1;
        sum += Q[k];
        if (arg < 0 || Q[k] > Q[arg]) arg = k;
    }
    if (arg >= 0) Q[arg] += ((int64_t)1 << 24) - sum;
}

/* Per-walker randomness of the learned proposal: two Philox calls. */
static void learned_draws(okey key, int phase, int comp, int64_t j, const uint32_t kd[2], uint32_t* V,
                          double* ure, double* uim)
{
    uint32_t a[4], b[4];
    uint32_t ctr[4] = {(uint32_t)key, (uint32_t)(key >> 32),   /* n <= 32: key < 2^64 */
                       (uint32_t)phase | ((uint32_t)comp << 1) | (KIND_LEARNED << 2),
                       (uint32_t)(((j >> 1) << 2) | ((j & 1) << 1))};
    orc_philox(ctr, kd, a);
    ctr[3] |= 1u;
    orc_philox(ctr, kd, b);
    *V = a[0] >> 8;
    *ure = (double)((((uint64_t)a[1]) << 21) | (a[2] >> 11)) * (1.0 / 9007199254740992.0);
    *uim = (double)((((uint64_t)b[0]) << 21) | (b[1] >> 11)) * (1.0 / 9007199254740992.0);
}

static int pop_reserve(pop* p, int64_t cap)
{
    if (p->cap >= cap) return ORC_OK;
    int64_t nc = p->cap ? p->cap : 16;
    while (nc < cap) nc *= 2;
    rec* nr = (rec*)realloc(p->r, (size_t)nc * sizeof(rec));
    if (!nr) return ORC_ERR_OOM;
    p->r = nr;
    p->cap = nc;
    return ORC_OK;
}

static int spawn_push(spawn_list* l, okey key, int64_t re, int64_t im, int noninit)
{
    if (l->len == l->cap) {
        int64_t nc = l->cap ? 2 * l->cap : 256;
        spawn_rec* ns = (spawn_rec*)realloc(l->s, (size_t)nc * sizeof(spawn_rec));
        if (!ns) return ORC_ERR_OOM;
        l->s = ns;
        l->cap = nc;
    }
    l->s[l->len].key = key;
    l->s[l->len].re = re;
    l->s[l->len].im = im;
    l->s[l->len].noninit = noninit;
    l->len++;
    return ORC_OK;
}

void* orc_state_new(const void* prob, int nseg, uint64_t seed, int integrator, int64_t init_min,
                    int64_t n_diag)
{
    if (!prob || nseg < 1) return NULL;
    state* s = (state*)calloc(1, sizeof(state));
    if (!s) return NULL;
    s->prob = (const problem*)prob;
    s->nseg = nseg;
    s->seed = seed;
    s->integrator = integrator;
    s->init_min = init_min;
    s->n_diag = n_diag;
    s->cur = (pop*)calloc((size_t)nseg, sizeof(pop));
    s->prev = (pop*)calloc((size_t)nseg, sizeof(pop));
    s->active = (unsigned char*)malloc((size_t)nseg);
    memset(s->active, 1, (size_t)nseg);
    return s;
}

void orc_state_free(void* sp)
{
    state* s = (state*)sp;
    if (!s) return;
    for (int i = 0; i < s->nseg; ++i) { free(s->cur[i].r); free(s->prev[i].r); }
    free(s->cur); free(s->prev); free(s->active);
    free(s->w1); free(s->b1); free(s->w2); free(s->b2); free(s->w3); free(s->b3); free(s->out_mask);
    free(s);
}

static int cmp_key(okey a, okey b) { return a < b ? -1 : (a > b ? 1 : 0); }

static int rec_cmp(const void* a, const void* b)
{
    return cmp_key(((const rec*)a)->key, ((const rec*)b)->key);
}

static int spawn_cmp(const void* a, const void* b)
{
    return cmp_key(((const spawn_rec*)a)->key, ((const spawn_rec*)b)->key);
}

/* N(0) := N^diag rho(0), each component stochastically rounded (reading R4).
 * The rounding draw of a component is keyed by the state's key: its bits
 * 0-63 in the first two counter words, 64-95 in the fourth, 96-119 in the
 * top 24 bits of the third (all zero for n <= 32). */
int orc_init(void* sp, int ne, const uint64_t* x, const uint64_t* y, const double* re,
             const double* im)
{
    state* s = (state*)sp;
    const int n = s->prob->n;
    for (int seg = 0; seg < s->nseg; ++seg) {
        uint32_t kd[2];
        derive_key(s->seed, 0, (uint32_t)seg, TAG_INIT, kd);
        pop* c = &s->cur[seg];
        c->len = 0;
        s->prev[seg].len = 0;
        if (pop_reserve(c, ne > 0 ? ne : 1) != ORC_OK) return ORC_ERR_OOM;
        for (int i = 0; i < ne; ++i) {
            const okey key = ((okey)x[i] << n) | y[i];
            int64_t v[2];
            for (int comp = 0; comp < 2; ++comp) {
                double val = (double)s->n_diag * (comp == 0 ? re[i] : im[i]);
                double fl = floor(val);
                double fr = val - fl;
                uint32_t ctr[4] = {(uint32_t)key, (uint32_t)(key >> 32),
                                   ((uint32_t)comp << 1) | (KIND_INIT << 2) | ((uint32_t)(key >> 96) << 8),
                                   (uint32_t)(key >> 64)};
                uint32_t w[4];
                orc_philox(ctr, kd, w);
                uint64_t r = ((uint64_t)w[1] << 32) | w[0];
                double u = (double)(r >> 11) * (1.0 / 9007199254740992.0);
                v[comp] = (int64_t)fl + (u < fr ? 1 : 0);
                if (v[comp] > INT32_MAX || v[comp] < -INT32_MAX) return ORC_ERR_POP_OVERFLOW;
            }
            if (v[0] == 0 && v[1] == 0) continue;
            c->r[c->len].key = key;
            c->r[c->len].re = (int32_t)v[0];
            c->r[c->len].im = (int32_t)v[1];
            c->len++;
        }
        qsort(c->r, (size_t)c->len, sizeof(rec), rec_cmp);
        for (int64_t i = 1; i < c->len; ++i)
            if (c->r[i].key == c->r[i - 1].key) return ORC_ERR_INVALID_ARG;
    }
    s->step = 0;
    s->t = 0.0;
    s->t_prev = 0.0;
    s->dt_last = 0.0;
    s->prev_valid = 0;
    return ORC_OK;
}

/* Population of vector seg (which 0: N(t), 1: N(t - dt)) from cnt records
 * |x[i]><y[i]| with values (re[i], im[i]); zero records are dropped. */
int orc_set_population_xy(void* sp, int seg, int which, int64_t cnt, const uint64_t* x, const uint64_t* y,
                          const int32_t* re, const int32_t* im)
{
    state* s = (state*)sp;
    if (seg < 0 || seg >= s->nseg) return ORC_ERR_INVALID_ARG;
    const int n = s->prob->n;
    const uint64_t lim = (((uint64_t)1) << n) - 1;
    pop* p = which ? &s->prev[seg] : &s->cur[seg];
    if (pop_reserve(p, cnt > 0 ? cnt : 1) != ORC_OK) return ORC_ERR_OOM;
    p->len = 0;
    for (int64_t i = 0; i < cnt; ++i) {
        if ((x[i] & ~lim) || (y[i] & ~lim)) return ORC_ERR_INVALID_ARG;
        if (re[i] == 0 && im[i] == 0) continue;
        p->r[p->len].key = ((okey)x[i] << n) | y[i];
        p->r[p->len].re = re[i];
        p->r[p->len].im = im[i];
        p->len++;
    }
    qsort(p->r, (size_t)p->len, sizeof(rec), rec_cmp);
    for (int64_t i = 1; i < p->len; ++i)
        if (p->r[i].key == p->r[i - 1].key) return ORC_ERR_INVALID_ARG;
    return ORC_OK;
}

/* The same with whole keys (x << n) | y (n <= 32). */
int orc_set_population(void* sp, int seg, int which, int64_t cnt, const uint64_t* keys,
                       const int32_t* re, const int32_t* im)
{
    state* s = (state*)sp;
    if (seg < 0 || seg >= s->nseg || s->prob->n > 32) return ORC_ERR_INVALID_ARG;
    const int n = s->prob->n;
    uint64_t* x = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)(cnt > 0 ? cnt : 1));
    uint64_t* y = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)(cnt > 0 ? cnt : 1));
    if (!x || !y) { free(x); free(y); return ORC_ERR_OOM; }
    for (int64_t i = 0; i < cnt; ++i) {
        x[i] = keys[i] >> n;
        y[i] = keys[i] & ((((uint64_t)1) << n) - 1);
    }
    const int rc = orc_set_population_xy(sp, seg, which, cnt, x, y, re, im);
    free(x);
    free(y);
    return rc;
}

/* Restrict orc_step to a subset of the vectors (each vector is independent,
 * so a subset evolves exactly as in the full run). */
int orc_set_active(void* sp, int seg, int on)
{
    state* s = (state*)sp;
    if (seg < 0 || seg >= s->nseg) return ORC_ERR_INVALID_ARG;
    s->active[seg] = on ? 1 : 0;
    return ORC_OK;
}

int orc_set_clock(void* sp, uint64_t step, double t, double t_prev, double dt_last, int prev_valid)
{
    state* s = (state*)sp;
    s->step = step;
    s->t = t;
    s->t_prev = t_prev;
    s->dt_last = dt_last;
    s->prev_valid = prev_valid;
    return ORC_OK;
}

void orc_get_clock(void* sp, uint64_t* step, double* tt)
{
    state* s = (state*)sp;
    *step = s->step;
    tt[0] = s->t;
    tt[1] = s->t_prev;
    tt[2] = s->dt_last;
    tt[3] = (double)s->prev_valid;
}

/*
 * Spawns of one parent [End Matter, spawn step].  phase 0: the population
 * N(t) (sign +1); phase 1: N(t - dt) in AB2 (sign -1).  Every spawned walker,
 * including one landing on the parent itself (the diagonal, "death/cloning"
 * element, which is one of the kl in the paper's sum), becomes one record.
 */
/* Value of the column at mask (0 if absent). */
static cint column_at(const column* c, uint64_t mask)
{
    int lo = 0, hi = c->len;
    while (lo < hi) {
        int mid = (lo + hi) / 2;
        if (c->e[mid].mask < mask) lo = mid + 1; else hi = mid;
    }
    cint z = {0, 0};
    if (lo < c->len && c->e[lo].mask == mask) z = c->e[lo].v;
    return z;
}

/*
 * The 52-bit draw T of walker j of component comp (0 real, 1 imaginary) of
 * the parent at rank r -- its index in the vector's key-sorted population --
 * in pass phase (0: N(t), 1: N(t - dt)), with the step's key kd (reading R3;
 * the paper names no generator).  The parent's walkers are numbered
 * w = 0 .. m - 1, real walkers first.  T = W << 20 | L, where W is a 32-bit
 * word -- for w = 0 and w = 1 word r % 4 of the rank group's call of level w
 * (one call serves walker w of four consecutive parents), for w >= 2 word
 * (w - 2) % 4 of the parent's call (w - 2) / 4 -- and L the top 20 bits of
 * word 0 of the walker's own call.  Every word comes from a distinct Philox
 * counter, so the T of all walkers are independent and uniform on [0, 2^52).
 */
static int64_t walker_T(const uint32_t kd[2], int64_t r, int phase, int comp, int64_t j, int64_t are)
{
    const int64_t w = (comp ? are : 0) + j;
    uint32_t o[4];
    uint32_t W;
    if (w <= 1) {
        const uint32_t ctr[4] = {(uint32_t)(r >> 2), (uint32_t)w, (uint32_t)phase | (KIND_GROUP << 2), 0u};
        orc_philox(ctr, kd, o);
        W = o[r & 3];
    } else {
        const uint32_t ctr[4] = {(uint32_t)r, (uint32_t)((w - 2) >> 2), (uint32_t)phase | (KIND_EXTRA << 2), 0u};
        orc_philox(ctr, kd, o);
        W = o[(w - 2) & 3];
    }
    const uint32_t ctr2[4] = {(uint32_t)r, (uint32_t)j, (uint32_t)phase | ((uint32_t)comp << 1) | (KIND_LOW << 2),
                              0u};
    orc_philox(ctr2, kd, o);
    return (int64_t)((((uint64_t)W) << 20) | (o[0] >> 12));
}

static int spawn_parent(const state* s, const rec* par, int64_t rank, int phase, double t, double dt_eff,
                        int sigma, const uint32_t kd[2], column* col, const column* st, spawn_list* out)
{
    const problem* p = s->prob;
    const int n = p->n;
    const uint64_t x = (uint64_t)(par->key >> n);
    const uint64_t y = (uint64_t)par->key & ((((uint64_t)1) << n) - 1);
    int rc = build_column(p, x, y, t, dt_eff, col);
    if (rc != ORC_OK) return rc;

    /* P = 2^52 * dt_eff * sum_kl (|Re L_kl| + |Im L_kl|); with the proposal the
     * attempt probability is the static sum instead */
    int64_t P = 0;
    if (s->proposal == 0) {
        for (int e = 0; e < col->len; ++e) {
            P += llabs(col->e[e].v.re) + llabs(col->e[e].v.im);
            if (P >= P_LIMIT) return ORC_ERR_DT_TOO_LARGE;
        }
    } else {
        for (int e = 0; e < st->len; ++e) {
            P += st->e[e].v.re;
            if (P >= P_LIMIT) return ORC_ERR_DT_TOO_LARGE;
        }
    }
    int64_t walkers = llabs((int64_t)par->re) + llabs((int64_t)par->im);
    int noninit = (s->init_min > 0 && walkers < s->init_min) ? 1 : 0;
    int64_t Qbuf[256];
    int64_t* Qw = Qbuf;
    if (s->proposal == 2) {
        if (st->len > 256) return ORC_ERR_INVALID_ARG;
        learned_weights(s, st, P, x, y, t, Qw);
    }

    for (int comp = 0; comp < 2; ++comp) {
        int64_t val = comp == 0 ? par->re : par->im;
        int64_t m = llabs(val);
        int64_t sg = val > 0 ? 1 : -1;
        for (int64_t j = 0; j < m; ++j) {
            int64_t T = walker_T(kd, rank, phase, comp, j, llabs((int64_t)par->re));
            if (T >= P) continue; /* this walker does not spawn */
            if (s->proposal == 2) {
                /* learned proposal: destination by Q, counts by the amplitude */
                uint32_t V;
                double ure, uim;
                learned_draws(par->key, phase, comp, j, kd, &V, &ure, &uim);
                int k = 0;
                int64_t cum = 0;
                for (k = 0; k < st->len; ++k) {
                    cum += Qw[k];
                    if ((int64_t)V < cum) break;
                }
                if (k >= st->len) continue;
                const cint v = column_at(col, st->e[k].mask);
                for (int chan = 0; chan < 2; ++chan) {
                    const int64_t w = llabs(chan ? v.im : v.re);
                    if (w == 0) continue;
                    const double A = ((double)w * 16777216.0) / ((double)Qw[k] * (double)P);
                    const double fl = floor(A);
                    int64_t cnt = (int64_t)fl + (((chan ? uim : ure) < A - fl) ? 1 : 0);
                    if (cnt == 0) continue;
                    int64_t dre = 0, dim = 0;
                    int64_t sv = sigma * sg * ((chan ? v.im : v.re) > 0 ? 1 : -1) * cnt;
                    if (chan == 0) { if (comp == 0) dre = sv; else dim = sv; }
                    else { if (comp == 0) dim = sv; else dre = -sv; }
                    rc = spawn_push(out, par->key ^ st->e[k].mask, dre, dim, noninit);
                    if (rc != ORC_OK) return rc;
                }
                continue;
            }
            if (s->proposal == 1) {
                /* destination by static weights (ascending mask), then the Re or
                 * Im channel by the exact element weights inside its interval */
                for (int e = 0; e < st->len; ++e) {
                    const int64_t sw = st->e[e].v.re;
                    if (T >= sw) {
                        T -= sw;
                        continue;
                    }
                    const cint v = column_at(col, st->e[e].mask);
                    const int64_t wr = llabs(v.re), wi = llabs(v.im);
                    int chan = T < wr ? 0 : (T < wr + wi ? 1 : -1);
                    if (chan >= 0) {
                        int64_t dre = 0, dim = 0;
                        if (chan == 0) {
                            int64_t sv = sigma * sg * (v.re > 0 ? 1 : -1);
                            if (comp == 0) dre = sv; else dim = sv;
                        } else {
                            int64_t sv = sigma * sg * (v.im > 0 ? 1 : -1);
                            if (comp == 0) dim = sv; else dre = -sv;
                        }
                        rc = spawn_push(out, par->key ^ st->e[e].mask, dre, dim, noninit);
                        if (rc != ORC_OK) return rc;
                    }
                    break;
                }
                continue;
            }
            /* multinomial over (destination, channel) in ascending mask order,
             * Re channel before Im channel */
            for (int e = 0; e < col->len; ++e) {
                int64_t wr = llabs(col->e[e].v.re);
                int64_t wi = llabs(col->e[e].v.im);
                int chan = -1;
                if (T < wr) chan = 0;
                else {
                    T -= wr;
                    if (T < wi) chan = 1;
                    else T -= wi;
                }
                if (chan < 0) continue;
                int64_t dre = 0, dim = 0;
                if (chan == 0) {
                    /* Re channel: sign s * sgn(Re L) */
                    int64_t sv = sigma * sg * (col->e[e].v.re > 0 ? 1 : -1);
                    if (comp == 0) dre = sv; else dim = sv;
                } else {
                    /* Im channel: sign i * s * sgn(Im L) */
                    int64_t sv = sigma * sg * (col->e[e].v.im > 0 ? 1 : -1);
                    if (comp == 0) dim = sv; else dre = -sv;
                }
                rc = spawn_push(out, par->key ^ col->e[e].mask, dre, dim, noninit);
                if (rc != ORC_OK) return rc;
                break;
            }
        }
    }
    return ORC_OK;
}

/* Annihilation [End Matter, annihilation step] with the initiator rule. */
static int annihilate(const pop* cur, spawn_list* sp, pop* next)
{
    qsort(sp->s, (size_t)sp->len, sizeof(spawn_rec), spawn_cmp);
    int rc = pop_reserve(next, cur->len + sp->len + 1);
    if (rc != ORC_OK) return rc;
    next->len = 0;
    int64_t i = 0, j = 0;
    while (i < cur->len || j < sp->len) {
        okey key;
        if (j >= sp->len || (i < cur->len && cur->r[i].key <= sp->s[j].key)) key = cur->r[i].key;
        else key = sp->s[j].key;
        int occupied = (i < cur->len && cur->r[i].key == key);
        int64_t re = 0, im = 0;
        if (occupied) { re = cur->r[i].re; im = cur->r[i].im; ++i; }
        while (j < sp->len && sp->s[j].key == key) {
            if (occupied || !sp->s[j].noninit) { re += sp->s[j].re; im += sp->s[j].im; }
            ++j;
        }
        if (re == 0 && im == 0) continue;
        if (re > INT32_MAX || re < -INT32_MAX || im > INT32_MAX || im < -INT32_MAX)
            return ORC_ERR_POP_OVERFLOW;
        next->r[next->len].key = key;
        next->r[next->len].re = (int32_t)re;
        next->r[next->len].im = (int32_t)im;
        next->len++;
    }
    return ORC_OK;
}

/*
 * nsteps steps of size dt.  Step i of this call uses L at t_i = t0 + i*dt,
 * where t0 is the clock at entry; an AB2 step's second pass uses L at the
 * time the previous step used.
 */
int orc_step(void* sp, double dt, int nsteps)
{
    state* s = (state*)sp;
    if (!(dt > 0.0) || nsteps < 0) return ORC_ERR_INVALID_ARG;
    column col = {0, 0, 0}, st_cur = {0, 0, 0}, st_prev = {0, 0, 0};
    spawn_list spl = {0, 0, 0};
    pop next = {0, 0, 0};
    int rc = ORC_OK;
    const double t0 = s->t;
    for (int it = 0; it < nsteps && rc == ORC_OK; ++it) {
        double t = t0 + (double)it * dt;
        int ab2 = (s->integrator == 1 && s->prev_valid && s->dt_last == dt);
        double dt_cur = ab2 ? dt * 1.5 : dt;
        double dt_prev = dt * 0.5;
        if (s->proposal) {
            rc = build_static(s->prob, t, dt_cur, &st_cur);
            if (rc == ORC_OK && ab2) rc = build_static(s->prob, s->t_prev, dt_prev, &st_prev);
            if (rc != ORC_OK) break;
        }
        for (int seg = 0; seg < s->nseg && rc == ORC_OK; ++seg) {
            if (!s->active[seg]) continue;
            uint32_t kd[2];
            derive_key(s->seed, s->step, (uint32_t)seg, TAG_STEP, kd);
            spl.len = 0;
            const pop* cur = &s->cur[seg];
            for (int64_t i = 0; i < cur->len && rc == ORC_OK; ++i)
                rc = spawn_parent(s, &cur->r[i], i, 0, t, dt_cur, 1, kd, &col, &st_cur, &spl);
            if (ab2) {
                const pop* prv = &s->prev[seg];
                for (int64_t i = 0; i < prv->len && rc == ORC_OK; ++i)
                    rc = spawn_parent(s, &prv->r[i], i, 1, s->t_prev, dt_prev, -1, kd, &col, &st_prev, &spl);
            }
            if (rc != ORC_OK) break;
            /* spawns from N(t - dt) that land on states unoccupied in N(t) are
             * treated like every other spawn: the initiator rule uses N(t). */
            rc = annihilate(cur, &spl, &next);
            if (rc != ORC_OK) break;
            /* rotate: prev <- cur, cur <- next */
            pop old_prev = s->prev[seg];
            s->prev[seg] = s->cur[seg];
            s->cur[seg] = next;
            next = old_prev;
        }
        if (rc != ORC_OK) break;
        s->t_prev = t;
        s->dt_last = dt;
        s->prev_valid = 1;
        s->step += 1;
        s->t = t0 + (double)(it + 1) * dt;
    }
    free(col.e);
    free(st_cur.e);
    free(st_prev.e);
    free(spl.s);
    free(next.r);
    return rc;
}

static void value_at_key(const pop* p, okey key, int64_t* re, int64_t* im);

/*
 * The value N(t + dt) of vector seg at one key after the next step of size dt
 * (what orc_step(dt, 1) would leave there), without stepping: every parent
 * that can spawn onto the key -- the occupied states key ^ mask of N(t) and,
 * in an AB2 step, of N(t - dt), for every destination mask with a nonzero
 * static weight -- replays its walkers exactly as in the step (spawn_parent,
 * same ranks and draws), and the spawns landing on the key are annihilated
 * with N(t)'s value there under the initiator rule.  For checking sampled
 * outputs of a large step one key at a time.  out = (re, im).
 */
int orc_next_value_xy(void* sp, int seg, double dt, uint64_t x, uint64_t y, int64_t out[2])
{
    state* s = (state*)sp;
    if (seg < 0 || seg >= s->nseg || !(dt > 0.0)) return ORC_ERR_INVALID_ARG;
    const okey key = ((okey)x << s->prob->n) | y;
    const double t = s->t;
    const int ab2 = (s->integrator == 1 && s->prev_valid && s->dt_last == dt);
    const double dt_cur = ab2 ? dt * 1.5 : dt;
    uint32_t kd[2];
    derive_key(s->seed, s->step, (uint32_t)seg, TAG_STEP, kd);
    column col = {0, 0, 0}, st_cur = {0, 0, 0}, st_prev = {0, 0, 0}, m_cur = {0, 0, 0}, m_prev = {0, 0, 0};
    spawn_list spl = {0, 0, 0};
    int rc = build_static(s->prob, t, dt_cur, &m_cur);
    if (rc == ORC_OK && ab2) rc = build_static(s->prob, s->t_prev, dt * 0.5, &m_prev);
    if (rc == ORC_OK && s->proposal) {
        rc = build_static(s->prob, t, dt_cur, &st_cur);
        if (rc == ORC_OK && ab2) rc = build_static(s->prob, s->t_prev, dt * 0.5, &st_prev);
    }
    int64_t re = 0, im = 0, cre = 0, cim = 0;
    const pop* cur = &s->cur[seg];
    value_at_key(cur, key, &cre, &cim);
    const int occupied = cre != 0 || cim != 0;
    for (int phase = 0; phase < (ab2 ? 2 : 1) && rc == ORC_OK; ++phase) {
        const pop* src = phase ? &s->prev[seg] : cur;
        const column* masks = phase ? &m_prev : &m_cur;
        for (int e = 0; e < masks->len && rc == ORC_OK; ++e) {
            const okey pk = key ^ masks->e[e].mask;
            /* the parent's rank: its index in the sorted population */
            int64_t lo = 0, hi = src->len;
            while (lo < hi) {
                const int64_t mid = (lo + hi) / 2;
                if (src->r[mid].key < pk) lo = mid + 1; else hi = mid;
            }
            if (lo >= src->len || src->r[lo].key != pk) continue;
            spl.len = 0;
            rc = phase ? spawn_parent(s, &src->r[lo], lo, 1, s->t_prev, dt * 0.5, -1, kd, &col, &st_prev, &spl)
                       : spawn_parent(s, &src->r[lo], lo, 0, t, dt_cur, 1, kd, &col, &st_cur, &spl);
            for (int64_t j = 0; j < spl.len && rc == ORC_OK; ++j) {
                if (spl.s[j].key != key) continue;
                if (!occupied && spl.s[j].noninit) continue;
                re += spl.s[j].re;
                im += spl.s[j].im;
            }
        }
    }
    free(col.e);
    free(st_cur.e);
    free(st_prev.e);
    free(m_cur.e);
    free(m_prev.e);
    free(spl.s);
    out[0] = cre + re;
    out[1] = cim + im;
    return rc;
}

/* orc_next_value_xy at the key (x << n) | y given whole (n <= 32). */
int orc_next_value(void* sp, int seg, double dt, uint64_t key, int64_t out[2])
{
    state* s = (state*)sp;
    const int n = s->prob->n;
    if (n > 32) return ORC_ERR_INVALID_ARG;
    return orc_next_value_xy(sp, seg, dt, key >> n, key & ((((uint64_t)1) << n) - 1), out);
}

/* Spawn choice of the following steps: 0 exact |L|-weighted (the paper's),
 * 1 static-weight proposal (see the header). */
int orc_set_proposal(void* sp, int kind)
{
    state* s = (state*)sp;
    if (kind < 0 || kind > 2 || (kind == 2 && (!s->w1 || s->prob->n > 32))) return ORC_ERR_INVALID_ARG;
    s->proposal = kind;
    return ORC_OK;
}

/* Network of the learned proposal (weights copied): n_in = 2n + 1 inputs,
 * n_hidden <= 64, n_out destination masks; w1 is n_hidden x n_in, w2
 * n_hidden x n_hidden, w3 n_out x n_hidden, all row-major. */
int orc_set_mlp(void* sp, int n_in, int n_hidden, int n_out, const uint64_t* out_mask, const float* w1,
                const float* b1, const float* w2, const float* b2, const float* w3, const float* b3, float eps)
{
    state* s = (state*)sp;
    if (s->prob->n > 32 || n_in != 2 * s->prob->n + 1 || n_hidden < 1 || n_hidden > 64 || n_out < 1 || !(eps > 0.0f) || eps > 1.0f)
        return ORC_ERR_INVALID_ARG;
    s->mlp_in = n_in;
    s->mlp_hidden = n_hidden;
    s->mlp_out = n_out;
    s->eps = eps;
#define ORC_COPY(dst, src, cnt, T)                                       \
    do {                                                                 \
        free(dst);                                                       \
        dst = (T*)malloc(sizeof(T) * (size_t)(cnt));                     \
        if (!dst) return ORC_ERR_OOM;                                    \
        memcpy(dst, src, sizeof(T) * (size_t)(cnt));                     \
    } while (0)
    ORC_COPY(s->w1, w1, n_hidden * n_in, float);
    ORC_COPY(s->b1, b1, n_hidden, float);
    ORC_COPY(s->w2, w2, n_hidden * n_hidden, float);
    ORC_COPY(s->b2, b2, n_hidden, float);
    ORC_COPY(s->w3, w3, n_out * n_hidden, float);
    ORC_COPY(s->b3, b3, n_out, float);
    ORC_COPY(s->out_mask, out_mask, n_out, uint64_t);
#undef ORC_COPY
    return ORC_OK;
}

/* Sum over the diagonal records of vector seg of Re N_xx (-1)^(x_q), for
 * q = 0 .. n - 1 (out[q]): N^diag <Z_q> in the walker representation
 * [walker averaging, Eq. (3): rho = N / N^diag].  Bit q of x is qubit q. */
void orc_zsum(void* sp, int seg, int64_t* out)
{
    state* s = (state*)sp;
    const int n = s->prob->n;
    const pop* p = &s->cur[seg];
    const uint64_t ymask = (((uint64_t)1) << n) - 1;
    for (int q = 0; q < n; ++q) out[q] = 0;
    for (int64_t i = 0; i < p->len; ++i) {
        const uint64_t x = (uint64_t)(p->r[i].key >> n), y = (uint64_t)p->r[i].key & ymask;
        if (x != y) continue;
        for (int q = 0; q < n; ++q) out[q] += ((x >> q) & 1u) ? -(int64_t)p->r[i].re : (int64_t)p->r[i].re;
    }
}

/* Value of vector seg's N(t) at key (0 when unoccupied). */
static void value_at_key(const pop* p, okey key, int64_t* re, int64_t* im)
{
    int64_t lo = 0, hi = p->len;
    while (lo < hi) {
        const int64_t mid = (lo + hi) / 2;
        if (p->r[mid].key < key) lo = mid + 1; else hi = mid;
    }
    *re = 0;
    *im = 0;
    if (lo < p->len && p->r[lo].key == key) {
        *re = p->r[lo].re;
        *im = p->r[lo].im;
    }
}

/* ||N - N^dagger||_F^2 of vector seg's N(t), exactly (out[0] low and out[1]
 * high 64 bits) [End Matter on Hermiticity preservation: epsilon =
 * ||rho - rho^dagger||_F with rho = N / N^diag].  The sum runs over every
 * entry (x, y) where N or N^dagger is nonzero: each record's entry
 * N_xy - conj(N_yx), and the transposed entry -conj(N_xy) of every record
 * whose transposed key is unoccupied. */
void orc_antiherm(void* sp, int seg, uint64_t out[2])
{
    state* s = (state*)sp;
    const int n = s->prob->n;
    const pop* p = &s->cur[seg];
    const uint64_t ymask = (((uint64_t)1) << n) - 1;
    unsigned __int128 acc = 0;
    for (int64_t i = 0; i < p->len; ++i) {
        const uint64_t x = (uint64_t)(p->r[i].key >> n), y = (uint64_t)p->r[i].key & ymask;
        int64_t tre, tim;
        value_at_key(p, ((okey)y << n) | x, &tre, &tim);
        const int64_t dre = (int64_t)p->r[i].re - tre, dim = (int64_t)p->r[i].im + tim;
        acc += (unsigned __int128)((__int128)dre * dre) + (unsigned __int128)((__int128)dim * dim);
        if (tre == 0 && tim == 0) {
            /* the transposed entry is -conj(N_xy) */
            const int64_t a = p->r[i].re, b = p->r[i].im;
            acc += (unsigned __int128)((__int128)a * a) + (unsigned __int128)((__int128)b * b);
        }
    }
    out[0] = (uint64_t)acc;
    out[1] = (uint64_t)(acc >> 64);
}

/* ||S - S^dagger||_F^2 of the sum S = sum over the listed vectors of their
 * N(t), exactly (out[0] low, out[1] high 64 bits): the aggregated
 * anti-Hermiticity of replicas [End Matter on Hermiticity preservation, with
 * the replica aggregate of the Markovian circuit dynamics section].  Every
 * entry (x, y) where some listed vector holds (x, y) or (y, x) contributes
 * |S_xy - conj(S_yx)|^2. */
void orc_antiherm_sum(void* sp, const int32_t* segs, int count, uint64_t out[2])
{
    state* s = (state*)sp;
    const int n = s->prob->n;
    const uint64_t ymask = (((uint64_t)1) << n) - 1;
    unsigned __int128 acc = 0;
    for (int a = 0; a < count; ++a) {
        const pop* p = &s->cur[segs[a]];
        for (int64_t i = 0; i < p->len; ++i) {
            const okey key = p->r[i].key;
            const okey tkey = ((key & ymask) << n) | (key >> n);
            /* visit each entry once: (x, y) from the first listed vector that holds it, and
             * (y, x) from there too when no listed vector holds (y, x) */
            int first = 1;
            for (int b = 0; b < a && first; ++b) {
                int64_t re, im;
                value_at_key(&s->cur[segs[b]], key, &re, &im);
                if (re != 0 || im != 0) first = 0;
            }
            if (!first) continue;
            int64_t sre = 0, sim = 0, tre = 0, tim = 0;
            int t_held = 0;
            for (int b = 0; b < count; ++b) {
                int64_t re, im;
                value_at_key(&s->cur[segs[b]], key, &re, &im);
                sre += re;
                sim += im;
                value_at_key(&s->cur[segs[b]], tkey, &re, &im);
                tre += re;
                tim += im;
                if (re != 0 || im != 0) t_held = 1;
            }
            const int64_t dre = sre - tre, dim = sim + tim;
            acc += (unsigned __int128)((__int128)dre * dre) + (unsigned __int128)((__int128)dim * dim);
            if (tkey != key && !t_held)   /* the transposed entry -conj(S_xy) */
                acc += (unsigned __int128)((__int128)sre * sre) + (unsigned __int128)((__int128)sim * sim);
        }
    }
    out[0] = (uint64_t)acc;
    out[1] = (uint64_t)(acc >> 64);
}

/* walker_T, exported for the tests of the draws' distribution. */
int64_t orc_walker_T(const uint32_t kd[2], int64_t r, int phase, int comp, int64_t j, int64_t are)
{
    return walker_T(kd, r, phase, comp, j, are);
}

/* The learned proposal's e^x (mlp_exp), exported for its accuracy test. */
float orc_mlp_exp(float x) { return mlp_exp(x); }

/* Integer proposal weights of the learned proposal (learned_weights) for the
 * source |x><y| under the static column of dt_eff L(t): up to cap
 * destinations in ascending mask order (mask[k], Q[k]), *p_att the attempt
 * weight (sum of the static weights).  Returns the number of destinations or
 * a negative error.  Exported for the tests of the network's forward pass. */
int orc_learned_q(void* sp, double t, double dt_eff, uint64_t x, uint64_t y, int cap, uint64_t* mask,
                  int64_t* Q, int64_t* p_att)
{
    state* s = (state*)sp;
    if (!s->w1 || s->prob->n > 32) return ORC_ERR_INVALID_ARG;
    column st = {0, 0, 0};
    int rc = build_static(s->prob, t, dt_eff, &st);
    if (rc != ORC_OK) { free(st.e); return rc; }
    if (st.len > 256 || st.len > cap) { free(st.e); return ORC_ERR_INVALID_ARG; }
    int64_t P = 0;
    for (int e = 0; e < st.len; ++e) P += st.e[e].v.re;
    int64_t Qw[256];
    learned_weights(s, &st, P, x, y, t, Qw);
    for (int e = 0; e < st.len; ++e) {
        mask[e] = (uint64_t)st.e[e].mask;
        Q[e] = Qw[e];
    }
    *p_att = P;
    const int len = st.len;
    free(st.e);
    return len;
}

int64_t orc_count(void* sp, int seg, int which)
{
    state* s = (state*)sp;
    if (seg < 0 || seg >= s->nseg) return -1;
    return which ? s->prev[seg].len : s->cur[seg].len;
}

int orc_export(void* sp, int seg, int which, uint64_t* keys, int32_t* re, int32_t* im)
{
    state* s = (state*)sp;
    if (seg < 0 || seg >= s->nseg || s->prob->n > 32) return ORC_ERR_INVALID_ARG;
    const pop* p = which ? &s->prev[seg] : &s->cur[seg];
    for (int64_t i = 0; i < p->len; ++i) {
        keys[i] = (uint64_t)p->r[i].key;
        re[i] = p->r[i].re;
        im[i] = p->r[i].im;
    }
    return ORC_OK;
}

/* The population as bit strings: record i is |x[i]><y[i]| (any n). */
int orc_export_xy(void* sp, int seg, int which, uint64_t* x, uint64_t* y, int32_t* re, int32_t* im)
{
    state* s = (state*)sp;
    if (seg < 0 || seg >= s->nseg) return ORC_ERR_INVALID_ARG;
    const int n = s->prob->n;
    const pop* p = which ? &s->prev[seg] : &s->cur[seg];
    for (int64_t i = 0; i < p->len; ++i) {
        x[i] = (uint64_t)(p->r[i].key >> n);
        y[i] = (uint64_t)p->r[i].key & ((((uint64_t)1) << n) - 1);
        re[i] = p->r[i].re;
        im[i] = p->r[i].im;
    }
    return ORC_OK;
}

/* K, N_tot = sum |re| + |im|, and N^diag = sum over x == y (re, im). */
void orc_stats(void* sp, int seg, int64_t out[4])
{
    state* s = (state*)sp;
    const int n = s->prob->n;
    const pop* p = &s->cur[seg];
    int64_t ntot = 0, dre = 0, dim = 0;
    const uint64_t ymask = (((uint64_t)1) << n) - 1;
    for (int64_t i = 0; i < p->len; ++i) {
        ntot += llabs((int64_t)p->r[i].re) + llabs((int64_t)p->r[i].im);
        if ((uint64_t)(p->r[i].key >> n) == ((uint64_t)p->r[i].key & ymask)) {
            dre += p->r[i].re;
            dim += p->r[i].im;
        }
    }
    out[0] = p->len;
    out[1] = ntot;
    out[2] = dre;
    out[3] = dim;
}
