// Evaluation of a compiled column program (qmc_types.h) at a source state
// |x><y|: the diagonal element and the weight P = 2^52 dt_eff sum over
// destinations of (|Re L| + |Im L|) [End Matter, spawn step], and the value of
// any destination.  Shared by the kernels and the host-side program check.
#pragma once
#include <stdint.h>

#include "qmc_types.h"

#ifdef __CUDACC__
#define QMC_HD __host__ __device__
#else
#define QMC_HD
#endif

namespace qmc {

QMC_HD inline int qmc_popc(uint32_t v)
{
#ifdef __CUDA_ARCH__
    return __popc(v);
#else
    return __builtin_popcount(v);
#endif
}

QMC_HD inline int64_t qmc_iabs64(int64_t v) { return v < 0 ? -v : v; }

// Index of the lowest set bit (v != 0).
QMC_HD inline int qmc_ctz(uint32_t v)
{
#ifdef __CUDA_ARCH__
    return __ffs(v) - 1;
#else
    return __builtin_ctz(v);
#endif
}

// ---------------------------------------------------------------------------
// Column program access
// ---------------------------------------------------------------------------
struct Prog {
    const ProgHeader* h;
    const SelfFam* sf;
    const SelfGen* sg;
    const Fam* fam;
    const Gen* gen;
    const GTerm* gt;
    const Entry* ent;
    const AffGroup* aff;
    const Run* run;
    const StatSlot* stat;
};

QMC_HD inline Prog prog_at(const uint8_t* base)
{
    Prog p;
    p.h = (const ProgHeader*)base;
    p.sf = (const SelfFam*)(base + p.h->off_selffam);
    p.sg = (const SelfGen*)(base + p.h->off_selfgen);
    p.fam = (const Fam*)(base + p.h->off_fam);
    p.gen = (const Gen*)(base + p.h->off_gen);
    p.gt = (const GTerm*)(base + p.h->off_gterm);
    p.ent = (const Entry*)(base + p.h->off_entry);
    p.aff = (const AffGroup*)(base + p.h->off_aff);
    p.run = (const Run*)(base + p.h->off_run);
    p.stat = (const StatSlot*)(base + p.h->off_stat);
    return p;
}

QMC_HD inline void gen_value(const Prog& p, int g, uint32_t x, uint32_t y,
                                          int64_t* vr, int64_t* vi)
{
    const Gen& G = p.gen[g];
    if (G.is_const) { *vr = G.cre; *vi = G.cim; return; }
    int64_t er = 0, ei = 0;
    for (int j = 0; j < G.count; ++j) {
        const GTerm& t = p.gt[G.first + j];
        const int par = (qmc_popc(x & t.zl) + qmc_popc(y & t.zr)) & 1;
        er += par ? -t.qre : t.qre;
        ei += par ? -t.qim : t.qim;
    }
    *vr = er;
    *vi = ei;
}

// Diagonal element (sre, sim) and P = 2^52 dt_eff sum_kl (|Re L| + |Im L|).
// Everything that depends on the state through per-qubit patterns is one
// affine form per member mask (three popcounts each); only multi-qubit
// parity terms are evaluated term by term.
QMC_HD inline int64_t column_weight(const Prog& p, uint32_t x, uint32_t y, int64_t* sre_out,
                                    int64_t* sim_out)
{
    const ProgHeader& h = *p.h;
    int64_t sre = h.self_const_re, sim = h.self_const_im;
    int64_t P = h.p_const;
    for (int i = 0; i < h.n_aff; ++i) {
        const AffGroup& g = p.aff[i];
        const int32_t cx = qmc_popc(x & g.members), cy = qmc_popc(y & g.members);
        const int32_t c11 = qmc_popc(x & y & g.members);
        sre += g.s0re + g.sare * cx + g.sbre * cy + g.scre * c11;
        sim += g.s0im + g.saim * cx + g.sbim * cy + g.scim * c11;
        P += g.f0 + g.fx * cx + g.fy * cy + g.f11 * c11;
    }
    for (int i = 0; i < h.n_selfgen; ++i) {
        const SelfGen g = p.sg[i];
        const int par = (qmc_popc(x & g.zl) + qmc_popc(y & g.zr)) & 1;
        sre += par ? -g.qre : g.qre;
        sim += par ? -g.qim : g.qim;
    }
    P += qmc_iabs64(sre) + qmc_iabs64(sim);
    for (int g = 0; g < h.n_nonconst_gen; ++g) {
        int64_t vr, vi;
        gen_value(p, g, x, y, &vr, &vi);
        P += qmc_iabs64(vr) + qmc_iabs64(vi);
    }
    *sre_out = sre;
    *sim_out = sim;
    return P;
}

QMC_HD inline void entry_value(const Prog& p, const Entry& e, uint32_t x, uint32_t y,
                                            int64_t sre, int64_t sim, int64_t* vr, int64_t* vi)
{
    if (e.kind == 0) {
        *vr = sre;
        *vi = sim;
    } else if (e.kind == 1) {
        const Fam& f = p.fam[e.idx & 0xFFFFu];
        const int q = (int)(e.idx >> 16);
        const int pi = (int)((((x >> q) & 1u) << 1) | ((y >> q) & 1u));
        *vr = f.tre[pi];
        *vi = f.tim[pi];
    } else {
        gen_value(p, (int)e.idx, x, y, vr, vi);
    }
}

// Destination of a walker with T < P: walking the column in canonical order
// (ascending mask, Re before Im within a destination), the (mask, channel)
// whose cumulative-weight interval holds T, and its value.  A family run is
// skipped whole by its summed weight (member weights depend on x_q, y_q
// only); inside the run members are visited in ascending q.  Returns false
// if T lies beyond the column (T >= P).
QMC_HD inline bool choose_destination(const Prog& p, uint32_t x, uint32_t y, int64_t sre, int64_t sim, int64_t T,
                                      uint64_t* mask, int* chan, int64_t* v)
{
    const int nr = p.h->n_run;
    for (int r = 0; r < nr; ++r) {
        const Run R = p.run[r];
        if (R.kind != 1u) {
            const Entry E = p.ent[R.idx];
            int64_t vr, vi;
            entry_value(p, E, x, y, sre, sim, &vr, &vi);
            const int64_t wr = qmc_iabs64(vr);
            if (T < wr) { *mask = E.mask_key; *chan = 0; *v = vr; return true; }
            T -= wr;
            const int64_t wi = qmc_iabs64(vi);
            if (T < wi) { *mask = E.mask_key; *chan = 1; *v = vi; return true; }
            T -= wi;
            continue;
        }
        const Fam& f = p.fam[R.idx];
        const uint32_t M = R.members;
        const uint32_t m3 = x & y & M, m2 = x & ~y & M, m1 = ~x & y & M, m0 = ~x & ~y & M;
        const int64_t W = f.a[3] * qmc_popc(m3) + f.a[2] * qmc_popc(m2) + f.a[1] * qmc_popc(m1) +
                          f.a[0] * qmc_popc(m0);
        if (T >= W) {
            T -= W;
            continue;
        }
        uint32_t nz = (f.a[3] ? m3 : 0u) | (f.a[2] ? m2 : 0u) | (f.a[1] ? m1 : 0u) | (f.a[0] ? m0 : 0u);
        while (nz) {
            const int q = qmc_ctz(nz);
            nz &= nz - 1u;
            const int pi = (int)((((x >> q) & 1u) << 1) | ((y >> q) & 1u));
            const int64_t wr = qmc_iabs64(f.tre[pi]);
            const uint64_t mk = ((uint64_t)((f.ab >> 1) & 1u) << (q + (int)R.shift)) | ((uint64_t)(f.ab & 1u) << q);
            if (T < wr) { *mask = mk; *chan = 0; *v = f.tre[pi]; return true; }
            T -= wr;
            const int64_t wi = qmc_iabs64(f.tim[pi]);
            if (T < wi) { *mask = mk; *chan = 1; *v = f.tim[pi]; return true; }
            T -= wi;
        }
        return false;
    }
    return false;
}

// Index of the destination entry with this mask, or -1.
QMC_HD inline int find_entry(const Prog& p, uint64_t mask)
{
    int lo = 0, hi = p.h->n_entry;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (p.ent[mid].mask_key < mask) lo = mid + 1; else hi = mid;
    }
    return (lo < p.h->n_entry && p.ent[lo].mask_key == mask) ? lo : -1;
}

// Element of the column at a destination mask (0 where the column has no
// entry).  The diagonal element needs the self-family forms.
QMC_HD inline void value_at_mask(const Prog& p, uint64_t mask, uint32_t x, uint32_t y, int64_t* vr, int64_t* vi)
{
    *vr = 0;
    *vi = 0;
    const int e = find_entry(p, mask);
    if (e < 0) return;
    int64_t sre = 0, sim = 0;
    if (p.ent[e].kind == 0u) (void)column_weight(p, x, y, &sre, &sim);
    entry_value(p, p.ent[e], x, y, sre, sim, vr, vi);
}

// Proposal spawning of an attempting walker with T in [0, p_att): the static
// slot whose interval holds T, then the Re channel if the offset inside it is
// below |Re L|, the Im channel if below |Re L| + |Im L|, else no spawn.
// Returns false for no spawn.
QMC_HD inline bool proposal_choose(const Prog& p, uint32_t x, uint32_t y, int64_t T, uint64_t* mask, int* chan,
                                   int64_t* v)
{
    int lo = 0, hi = p.h->n_stat;   // first slot with end > T
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (p.stat[mid].end > T) hi = mid; else lo = mid + 1;
    }
    if (lo >= p.h->n_stat) return false;
    const int64_t start = lo ? p.stat[lo - 1].end : 0;
    const int64_t U = T - start;
    int64_t vr, vi;
    value_at_mask(p, p.stat[lo].mask, x, y, &vr, &vi);
    const int64_t wr = qmc_iabs64(vr), wi = qmc_iabs64(vi);
    *mask = p.stat[lo].mask;
    if (U < wr) { *chan = 0; *v = vr; return true; }
    if (U < wr + wi) { *chan = 1; *v = vi; return true; }
    return false;
}

} // namespace qmc
