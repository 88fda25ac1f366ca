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

QMC_HD inline int qmc_popc(uint64_t v)
{
#ifdef __CUDA_ARCH__
    return __popcll(v);
#else
    return __builtin_popcountll(v);
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

QMC_HD inline int qmc_ctz(uint64_t v)
{
#ifdef __CUDA_ARCH__
    return __ffsll((long long)v) - 1;
#else
    return __builtin_ctzll(v);
#endif
}

// ---------------------------------------------------------------------------
// Column program access.  M is the qubit-mask type (uint32_t up to 32
// qubits, uint64_t above), K the key / destination-mask type (uint64_t or
// u128).  States are passed as their bit strings x, y of type M.
// ---------------------------------------------------------------------------
template <class M, class K>
struct ProgT {
    using mask_t = M;
    using key_t = K;
    const ProgHeader* h;
    const SelfFamT<M>* sf;
    const SelfGenT<M>* sg;
    const FamT<M>* fam;
    const GenT<K>* gen;
    const GTermT<M>* gt;
    const EntryT<K>* ent;
    const AffGroupT<M>* aff;
    const RunT<M>* run;
    const StatSlotT<K>* stat;
};

using Prog = ProgT<uint32_t, uint64_t>;
using WProg = ProgT<uint64_t, u128>;

template <class M, class K>
QMC_HD inline ProgT<M, K> prog_at_t(const uint8_t* base)
{
    ProgT<M, K> p;
    p.h = (const ProgHeader*)base;
    p.sf = (const SelfFamT<M>*)(base + p.h->off_selffam);
    p.sg = (const SelfGenT<M>*)(base + p.h->off_selfgen);
    p.fam = (const FamT<M>*)(base + p.h->off_fam);
    p.gen = (const GenT<K>*)(base + p.h->off_gen);
    p.gt = (const GTermT<M>*)(base + p.h->off_gterm);
    p.ent = (const EntryT<K>*)(base + p.h->off_entry);
    p.aff = (const AffGroupT<M>*)(base + p.h->off_aff);
    p.run = (const RunT<M>*)(base + p.h->off_run);
    p.stat = (const StatSlotT<K>*)(base + p.h->off_stat);
    return p;
}

QMC_HD inline Prog prog_at(const uint8_t* base) { return prog_at_t<uint32_t, uint64_t>(base); }
QMC_HD inline WProg wprog_at(const uint8_t* base) { return prog_at_t<uint64_t, u128>(base); }

template <class M, class K>
QMC_HD inline void gen_value(const ProgT<M, K>& p, int g, typename ProgT<M, K>::mask_t x,
                             typename ProgT<M, K>::mask_t y, int64_t* vr, int64_t* vi)
{
    const GenT<K>& G = p.gen[g];
    if (G.is_const) { *vr = G.cre; *vi = G.cim; return; }
    int64_t er = 0, ei = 0;
    for (int j = 0; j < G.count; ++j) {
        const GTermT<M>& t = p.gt[G.first + j];
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
template <class M, class K>
QMC_HD inline int64_t column_weight(const ProgT<M, K>& p, typename ProgT<M, K>::mask_t x,
                                    typename ProgT<M, K>::mask_t y, int64_t* sre_out, int64_t* sim_out)
{
    const ProgHeader& h = *p.h;
    int64_t sre = h.self_const_re, sim = h.self_const_im;
    int64_t P = h.p_const;
    for (int i = 0; i < h.n_aff; ++i) {
        const AffGroupT<M>& g = p.aff[i];
        const int32_t cx = qmc_popc(x & g.members), cy = qmc_popc(y & g.members);
        const int32_t c11 = qmc_popc(x & y & g.members);
        sre += g.s0re + g.sare * cx + g.sbre * cy + g.scre * c11;
        sim += g.s0im + g.saim * cx + g.sbim * cy + g.scim * c11;
        P += g.f0 + g.fx * cx + g.fy * cy + g.f11 * c11;
    }
    for (int i = 0; i < h.n_selfgen; ++i) {
        const SelfGenT<M> g = p.sg[i];
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

template <class M, class K>
QMC_HD inline void entry_value(const ProgT<M, K>& p, const EntryT<K>& e, typename ProgT<M, K>::mask_t x,
                               typename ProgT<M, K>::mask_t y, int64_t sre, int64_t sim, int64_t* vr, int64_t* vi)
{
    if (e.kind == 0) {
        *vr = sre;
        *vi = sim;
    } else if (e.kind == 1) {
        const FamT<M>& f = p.fam[e.idx & 0xFFFFu];
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
template <class M, class K>
QMC_HD inline bool choose_destination(const ProgT<M, K>& p, typename ProgT<M, K>::mask_t x,
                                      typename ProgT<M, K>::mask_t y, int64_t sre, int64_t sim, int64_t T,
                                      K* mask, int* chan, int64_t* v)
{
    const int nr = p.h->n_run;
    for (int r = 0; r < nr; ++r) {
        const RunT<M> R = p.run[r];
        if (R.kind != 1u) {
            const EntryT<K> E = p.ent[R.idx];
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
        const FamT<M>& f = p.fam[R.idx];
        const M mem = R.members;
        const M m3 = x & y & mem, m2 = x & ~y & mem, m1 = ~x & y & mem, m0 = ~x & ~y & mem;
        const int64_t W = f.a[3] * qmc_popc(m3) + f.a[2] * qmc_popc(m2) + f.a[1] * qmc_popc(m1) +
                          f.a[0] * qmc_popc(m0);
        if (T >= W) {
            T -= W;
            continue;
        }
        M nz = (f.a[3] ? m3 : (M)0) | (f.a[2] ? m2 : (M)0) | (f.a[1] ? m1 : (M)0) | (f.a[0] ? m0 : (M)0);
        while (nz) {
            const int q = qmc_ctz(nz);
            nz &= nz - (M)1;
            const int pi = (int)((((x >> q) & 1u) << 1) | ((y >> q) & 1u));
            const int64_t wr = qmc_iabs64(f.tre[pi]);
            const K mk = ((K)((f.ab >> 1) & 1u) << (q + (int)R.shift)) | ((K)(f.ab & 1u) << q);
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
template <class M, class K>
QMC_HD inline int find_entry(const ProgT<M, K>& p, typename ProgT<M, K>::key_t mask)
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
template <class M, class K>
QMC_HD inline void value_at_mask(const ProgT<M, K>& p, typename ProgT<M, K>::key_t mask,
                                 typename ProgT<M, K>::mask_t x, typename ProgT<M, K>::mask_t y, int64_t* vr,
                                 int64_t* vi)
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
template <class M, class K>
QMC_HD inline bool proposal_choose(const ProgT<M, K>& p, typename ProgT<M, K>::mask_t x,
                                   typename ProgT<M, K>::mask_t y, int64_t T, K* mask, int* chan, int64_t* v)
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
