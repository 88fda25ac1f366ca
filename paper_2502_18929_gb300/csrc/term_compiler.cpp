// Host term compiler [Eq. (1), Eq. (2)].
//
// Expansion (per step, pass scale dt_eff; every expanded coefficient is
// rounded on its own to the 2^-52 grid, so element sums are exact integers):
//   -i[H, rho], term h P with s = rate(t) dt_eff, v = h s:
//       (-i v) P rho         and   (+i v) rho P
//   gamma(t) (L rho L^dag - 1/2 L^dag L rho - 1/2 rho L^dag L),
//   L = sum_a l_a P_a, s = gamma(t) dt_eff, hs = -s/2, for ordered pairs (a, b),
//   z = l_a conj(l_b):
//       (s z) P_a rho P_b
//       (hs conj z) (P_a P_b) rho   and   (hs conj z) rho (P_a P_b)
// A term c P_L rho P_R sends |x><y| to
//   c i^{nY(L)} (-i)^{nY(R)} (-1)^{popc(x & zL) + popc(y & zR)} |x^xL><y^xR|,
// nY = number of Y letters; the phase is folded into the stored Q'.
//
// Compiled with -ffp-contract=off: each product and sum above is rounded
// exactly as written.
#include "term_compiler.h"

#include <algorithm>
#include <array>
#include <cmath>
#include <cstring>
#include <map>
#include <tuple>
#include <utility>

#include "qmc_types.h"

namespace qmc {
namespace {

constexpr double kOne52 = 4503599627370496.0;       // 2^52
constexpr double kLimit62 = 4611686018427387904.0;  // 2^62

// One expanded term c P_L rho P_R: X and Z masks of both strings (M is the
// qubit-mask type, uint32_t up to 32 qubits and uint64_t above).
template <class M>
struct RawT {
    M xl, zl, xr, zr;
    int64_t qre, qim;
};

inline int popc(uint32_t v) { return __builtin_popcount(v); }
inline int popc(uint64_t v) { return __builtin_popcountll(v); }
inline int ctz(uint32_t v) { return __builtin_ctz(v); }
inline int ctz(uint64_t v) { return __builtin_ctzll(v); }

inline void rot(int64_t* re, int64_t* im, int k)
{
    int64_t a = *re, b = *im;
    switch (k & 3) {
    case 0: break;
    case 1: *re = -b; *im = a; break;
    case 2: *re = -a; *im = -b; break;
    default: *re = b; *im = -a; break;
    }
}

int quantise(double re, double im, int64_t* qre, int64_t* qim)
{
    double a = re * kOne52, b = im * kOne52;
    if (!(std::fabs(a) < kLimit62) || !(std::fabs(b) < kLimit62)) return QMC_ERR_COEF_RANGE;
    *qre = (int64_t)std::nearbyint(a);
    *qim = (int64_t)std::nearbyint(b);
    return QMC_OK;
}

double rate_value(const Schedule& s, int id, double t)
{
    const qmc_rate& r = s.rates[id];
    if (r.kind == QMC_RATE_COS) return r.a * std::cos(r.b * t + r.c);
    return r.a;
}

bool window_on(const Schedule& s, int id, double t)
{
    if (id < 0) return true;
    return s.windows[id].t0 <= t && t < s.windows[id].t1;
}

// P_a P_b = i^k P_c for Hermitian Pauli strings: on each qubit XY = iZ,
// YZ = iX, ZX = iY and the reverse orders give -i (i^3); counted over all
// qubits at once from the masks of each letter.
template <class M>
void pauli_mul(int n, M xa, M za, M xb, M zb, M* xc, M* zc, int* k)
{
    (void)n;
    const M Xa = xa & ~za, Ya = xa & za, Za = za & ~xa;
    const M Xb = xb & ~zb, Yb = xb & zb, Zb = zb & ~xb;
    const int fwd = popc((M)((Xa & Yb) | (Ya & Zb) | (Za & Xb)));
    const int rev = popc((M)((Ya & Xb) | (Za & Yb) | (Xa & Zb)));
    *xc = xa ^ xb;
    *zc = za ^ zb;
    *k = (fwd + 3 * rev) & 3;
}

template <class M>
int expand(const Schedule& s, double t, double dt_eff, std::vector<RawT<M>>* out)
{
    out->clear();
    int rc;
    for (const qmc_ham_term& h : s.ham) {
        if (!window_on(s, h.window_id, t)) continue;
        double sc = rate_value(s, h.rate_id, t) * dt_eff;
        double v = h.h * sc;
        const M xm = (M)h.xm, zm = (M)h.zm;
        int ny = popc(xm & zm);
        RawT<M> a{xm, zm, 0, 0, 0, 0}, b{0, 0, xm, zm, 0, 0};
        if ((rc = quantise(0.0, -v, &a.qre, &a.qim)) != QMC_OK) return rc;
        if ((rc = quantise(0.0, v, &b.qre, &b.qim)) != QMC_OK) return rc;
        rot(&a.qre, &a.qim, ny);
        rot(&b.qre, &b.qim, 4 - (ny & 3));
        out->push_back(a);
        out->push_back(b);
    }
    for (const qmc_lindblad& L : s.lind) {
        if (!window_on(s, L.window_id, t)) continue;
        double sc = rate_value(s, L.rate_id, t) * dt_eff;
        double hs = -0.5 * sc;
        for (int ia = 0; ia < L.count; ++ia) {
            const qmc_pauli_coef& la = s.coefs[L.first + ia];
            for (int ib = 0; ib < L.count; ++ib) {
                const qmc_pauli_coef& lb = s.coefs[L.first + ib];
                double zre = la.re * lb.re + la.im * lb.im;
                double zim = la.im * lb.re - la.re * lb.im;
                const M xa = (M)la.xm, za = (M)la.zm;
                const M xb = (M)lb.xm, zb = (M)lb.zm;
                RawT<M> j{xa, za, xb, zb, 0, 0};
                if ((rc = quantise(sc * zre, sc * zim, &j.qre, &j.qim)) != QMC_OK) return rc;
                rot(&j.qre, &j.qim, popc(xa & za) - popc(xb & zb) + 4);
                out->push_back(j);
                int64_t cre, cim;
                if ((rc = quantise(hs * zre, -(hs * zim), &cre, &cim)) != QMC_OK) return rc;
                M xc, zc;
                int k;
                pauli_mul(s.n, xa, za, xb, zb, &xc, &zc, &k);
                int nyc = popc(xc & zc);
                RawT<M> l{xc, zc, 0, 0, cre, cim}, r{0, 0, xc, zc, cre, cim};
                rot(&l.qre, &l.qim, k + nyc);
                rot(&r.qre, &r.qim, k - nyc + 4);
                out->push_back(l);
                out->push_back(r);
            }
        }
    }
    return QMC_OK;
}

// Copy count records into the blob with their padding bytes zeroed (with
// 64-bit masks and 128-bit keys several records have padding), so a program's
// bytes depend on its contents alone and equal programs compare equal.
template <typename T>
void put(std::vector<uint8_t>* blob, size_t at, const T* src, size_t count)
{
    for (size_t i = 0; i < count; ++i) {
        T rec = src[i];
        __builtin_clear_padding(&rec);
        std::memcpy(blob->data() + at + i * sizeof(T), &rec, sizeof(T));
    }
}

template <size_t A>
size_t align_up(size_t v) { return (v + (A - 1)) & ~(A - 1); }

template <class M, class K, size_t A>
int build_program_t(const Schedule& s, double t, double dt_eff, std::vector<uint8_t>* blob);

} // namespace

int validate_schedule(const Schedule& s, std::string* why)
{
    const uint64_t lim = (s.n >= 64) ? ~0ull : ((1ull << s.n) - 1);
    auto bad = [&](const char* m) { if (why) *why = m; return QMC_ERR_INVALID_ARG; };
    for (const auto& r : s.rates)
        if (r.kind != QMC_RATE_CONST && r.kind != QMC_RATE_COS) return bad("unknown rate kind");
    for (const auto& w : s.windows)
        if (!(w.t0 <= w.t1)) return bad("window with t0 > t1");
    for (const auto& h : s.ham) {
        if (h.rate_id < 0 || h.rate_id >= (int)s.rates.size()) return bad("hamiltonian rate id");
        if (h.window_id < -1 || h.window_id >= (int)s.windows.size()) return bad("hamiltonian window id");
        if ((h.xm & ~lim) || (h.zm & ~lim)) return bad("hamiltonian mask beyond n qubits");
    }
    for (const auto& L : s.lind) {
        if (L.rate_id < 0 || L.rate_id >= (int)s.rates.size()) return bad("lindblad rate id");
        if (L.window_id < -1 || L.window_id >= (int)s.windows.size()) return bad("lindblad window id");
        if (L.first < 0 || L.count < 1 || L.first + L.count > (int)s.coefs.size())
            return bad("lindblad coefficient range");
    }
    for (const auto& c : s.coefs)
        if ((c.xm & ~lim) || (c.zm & ~lim)) return bad("lindblad mask beyond n qubits");
    return QMC_OK;
}

double spawn_prob_bound(const Schedule& s, double t, double dt_eff)
{
    std::vector<RawT<uint64_t>> raw;
    if (expand(s, t, dt_eff, &raw) != QMC_OK) return INFINITY;
    double acc = 0.0;
    for (const RawT<uint64_t>& r : raw) acc += (std::fabs((double)r.qre) + std::fabs((double)r.qim)) / kOne52;
    return acc;
}

int build_program(const Schedule& s, double t, double dt_eff, std::vector<uint8_t>* blob)
{
    if (s.n <= 32) return build_program_t<uint32_t, uint64_t, 8>(s, t, dt_eff, blob);
    return build_program_t<uint64_t, u128, 16>(s, t, dt_eff, blob);
}

namespace {

// The program of one step and pass with qubit masks M and keys K; sections
// aligned to A bytes (16 for 128-bit keys).
template <class M, class K, size_t A>
int build_program_t(const Schedule& s, double t, double dt_eff, std::vector<uint8_t>* blob)
{
    using SelfFam = SelfFamT<M>;
    using SelfGen = SelfGenT<M>;
    using Fam = FamT<M>;
    using AffGroup = AffGroupT<M>;
    using Gen = GenT<K>;
    using GTerm = GTermT<M>;
    using Entry = EntryT<K>;
    using Run = RunT<M>;
    using StatSlot = StatSlotT<K>;
    const int n = s.n;
    std::vector<RawT<M>> raw;
    int rc = expand(s, t, dt_eff, &raw);
    if (rc != QMC_OK) return rc;

    // group by destination mask, merge equal parity terms (exact sums): the
    // expanded terms sorted by (destination mask, zl, zr), equal keys summed;
    // a group is a stretch of one mask, in ascending mask order
    struct KeyedTerm {
        K mk;
        M zl, zr;
        int64_t qre, qim;
    };
    std::vector<KeyedTerm> sorted;
    sorted.reserve(raw.size());
    for (const RawT<M>& r : raw) sorted.push_back(KeyedTerm{((K)r.xl << n) | (K)r.xr, r.zl, r.zr, r.qre, r.qim});
    std::sort(sorted.begin(), sorted.end(), [](const KeyedTerm& a, const KeyedTerm& b) {
        if (a.mk != b.mk) return a.mk < b.mk;
        if (a.zl != b.zl) return a.zl < b.zl;
        return a.zr < b.zr;
    });
    std::vector<KeyedTerm> merged;
    merged.reserve(sorted.size());
    for (const KeyedTerm& r : sorted) {
        if (!merged.empty() && merged.back().mk == r.mk && merged.back().zl == r.zl && merged.back().zr == r.zr) {
            merged.back().qre += r.qre;
            merged.back().qim += r.qim;
        } else {
            merged.push_back(r);
        }
    }
    size_t g0 = 0;   // merged[0, g0): the diagonal group (mask 0)
    while (g0 < merged.size() && merged[g0].mk == (K)0) ++g0;

    ProgHeader hdr;
    std::memset(&hdr, 0, sizeof(hdr));
    std::vector<SelfFam> selffam;
    std::vector<SelfGen> selfgen;
    std::vector<Fam> fams;
    std::vector<Gen> gen_nc, gen_c;
    std::vector<std::vector<GTerm>> gen_terms_nc, gen_terms_c;

    // diagonal (self) group
    {
        std::map<std::tuple<uint32_t, int64_t, int64_t>, M> sf; // (type, q) -> members
        {
            for (size_t i = 0; i < g0; ++i) {
                const M zl = merged[i].zl, zr = merged[i].zr;
                int64_t qre = merged[i].qre, qim = merged[i].qim;
                if (qre == 0 && qim == 0) continue;
                if (zl == 0 && zr == 0) {
                    hdr.self_const_re += qre;
                    hdr.self_const_im += qim;
                } else if (zr == 0 && popc(zl) == 1) {
                    sf[{0u, qre, qim}] |= zl;
                } else if (zl == 0 && popc(zr) == 1) {
                    sf[{1u, qre, qim}] |= zr;
                } else if (zl == zr && popc(zl) == 1) {
                    sf[{2u, qre, qim}] |= zl;
                } else {
                    selfgen.push_back(SelfGen{zl, zr, qre, qim});
                }
            }
        }
        for (const auto& kv : sf)
            selffam.push_back(SelfFam{kv.second, std::get<0>(kv.first), std::get<1>(kv.first),
                                      std::get<2>(kv.first)});
    }

    // off-diagonal groups: single-qubit families or generic groups
    std::map<std::array<int64_t, 9>, M> famkeys; // (ab, tre[4], tim[4]) -> members
    for (size_t ga = g0, gb = g0; ga < merged.size(); ga = gb) {
        const K mk = merged[ga].mk;
        while (gb < merged.size() && merged[gb].mk == mk) ++gb;
        const M xl = (M)(mk >> n), xr = (M)(mk & (((K)1 << n) - 1));
        const M qm = xl | xr;
        bool single = popc(qm) == 1;
        std::vector<GTerm> terms;
        for (size_t i = ga; i < gb; ++i) {
            const KeyedTerm& kt = merged[i];
            if (kt.qre == 0 && kt.qim == 0) continue;
            terms.push_back(GTerm{kt.zl, kt.zr, kt.qre, kt.qim});
            if ((kt.zl & ~qm) || (kt.zr & ~qm)) single = false;
        }
        if (terms.empty()) continue;
        if (single) {
            int q = ctz(qm);
            int64_t tre[4] = {0, 0, 0, 0}, tim[4] = {0, 0, 0, 0};
            for (int pi = 0; pi < 4; ++pi) {
                int xq = pi >> 1, yq = pi & 1;
                for (const GTerm& g : terms) {
                    int par = (xq & ((g.zl >> q) & 1)) ^ (yq & ((g.zr >> q) & 1));
                    tre[pi] += par ? -g.qre : g.qre;
                    tim[pi] += par ? -g.qim : g.qim;
                }
            }
            bool allzero = true;
            for (int pi = 0; pi < 4; ++pi) allzero = allzero && tre[pi] == 0 && tim[pi] == 0;
            if (allzero) continue;
            uint32_t ab = ((xl != 0) ? 2u : 0u) | ((xr != 0) ? 1u : 0u);
            const std::array<int64_t, 9> key = {(int64_t)ab, tre[0], tre[1], tre[2], tre[3],
                                                tim[0], tim[1], tim[2], tim[3]};
            famkeys[key] |= qm;
            continue;
        }
        bool is_const = true;
        for (const GTerm& g : terms) is_const = is_const && g.zl == 0 && g.zr == 0;
        Gen G{};
        G.mask_key = mk;
        G.is_const = is_const ? 1 : 0;
        if (is_const) {
            for (const GTerm& g : terms) { G.cre += g.qre; G.cim += g.qim; }
            if (G.cre == 0 && G.cim == 0) continue;
            gen_c.push_back(G);
            gen_terms_c.push_back(terms);
        } else {
            gen_nc.push_back(G);
            gen_terms_nc.push_back(terms);
        }
    }
    for (const auto& kv : famkeys) {
        Fam f{};
        f.members = kv.second;
        f.ab = (uint32_t)kv.first[0];
        for (int pi = 0; pi < 4; ++pi) {
            f.tre[pi] = kv.first[1 + pi];
            f.tim[pi] = kv.first[5 + pi];
            f.a[pi] = std::llabs(f.tre[pi]) + std::llabs(f.tim[pi]);
        }
        fams.push_back(f);
    }

    // affine forms per member mask (self families and families)
    std::map<M, AffGroup> aff;
    auto group = [&](M mem) -> AffGroup& {
        auto it = aff.find(mem);
        if (it == aff.end()) {
            AffGroup g{};
            g.members = mem;
            it = aff.emplace(mem, g).first;
        }
        return it->second;
    };
    for (const SelfFam& f : selffam) {
        AffGroup& g = group(f.members);
        const int64_t m = popc(f.members);
        g.s0re += f.qre * m;
        g.s0im += f.qim * m;
        if (f.type == 0 || f.type == 2) { g.sare -= 2 * f.qre; g.saim -= 2 * f.qim; }
        if (f.type == 1 || f.type == 2) { g.sbre -= 2 * f.qre; g.sbim -= 2 * f.qim; }
        if (f.type == 2) { g.scre += 4 * f.qre; g.scim += 4 * f.qim; }
    }
    for (const Fam& f : fams) {
        AffGroup& g = group(f.members);
        const int64_t m = popc(f.members);
        // pi = 2 x_q + y_q: a[0] (00), a[1] (01), a[2] (10), a[3] (11)
        g.f0 += f.a[0] * m;
        g.fx += f.a[2] - f.a[0];
        g.fy += f.a[1] - f.a[0];
        g.f11 += f.a[3] - f.a[2] - f.a[1] + f.a[0];
    }
    std::vector<AffGroup> affs;
    for (const auto& kv : aff) affs.push_back(kv.second);

    // Upper bound of P over all states (triangle inequality across groups; each
    // affine form maximised exactly over its feasible counts).  Used only to
    // skip the exact weight when a walker's draw already exceeds it.
    {
        int64_t b = std::llabs(hdr.self_const_re) + std::llabs(hdr.self_const_im);
        for (const Gen& g : gen_c) b += std::llabs(g.cre) + std::llabs(g.cim);
        for (const AffGroup& g : affs) {
            // |er| + |ei| + f is convex in the counts (cx, cy, c11), whose
            // feasible values are the integer points of the simplex spanned by
            // the four ways all m members share one bit pattern (x_q, y_q):
            // the maximum is at one of its corners.
            const int m = popc(g.members);
            const int corner[4][3] = {{0, 0, 0}, {0, m, 0}, {m, 0, 0}, {m, m, m}};
            int64_t best = 0;
            for (const auto& c : corner) {
                const int cx = c[0], cy = c[1], c11 = c[2];
                const int64_t er = g.s0re + g.sare * cx + g.sbre * cy + g.scre * c11;
                const int64_t ei = g.s0im + g.saim * cx + g.sbim * cy + g.scim * c11;
                const int64_t f = g.f0 + g.fx * cx + g.fy * cy + g.f11 * c11;
                best = std::max<int64_t>(best, (int64_t)(std::llabs(er) + std::llabs(ei)) + f);
            }
            b += best;
        }
        for (const SelfGen& g : selfgen) b += std::llabs(g.qre) + std::llabs(g.qim);
        for (size_t i = 0; i < gen_nc.size(); ++i)
            for (const GTerm& g : gen_terms_nc[i]) b += std::llabs(g.qre) + std::llabs(g.qim);
        hdr.p_bound = b;
    }

    std::vector<Gen> gens;
    std::vector<GTerm> gterms;
    hdr.n_nonconst_gen = (int32_t)gen_nc.size();
    for (size_t i = 0; i < gen_nc.size(); ++i) {
        Gen g = gen_nc[i];
        g.first = (int32_t)gterms.size();
        g.count = (int32_t)gen_terms_nc[i].size();
        gterms.insert(gterms.end(), gen_terms_nc[i].begin(), gen_terms_nc[i].end());
        gens.push_back(g);
    }
    for (size_t i = 0; i < gen_c.size(); ++i) {
        Gen g = gen_c[i];
        g.first = (int32_t)gterms.size();
        g.count = (int32_t)gen_terms_c[i].size();
        gterms.insert(gterms.end(), gen_terms_c[i].begin(), gen_terms_c[i].end());
        hdr.p_const += std::llabs(g.cre) + std::llabs(g.cim);
        gens.push_back(g);
    }

    // destinations in ascending mask order (the multinomial's canonical order)
    std::vector<Entry> entries;
    entries.push_back(Entry{(K)0, 0u, 0u});
    for (size_t f = 0; f < fams.size(); ++f) {
        M m = fams[f].members;
        while (m) {
            int q = ctz(m);
            m &= m - 1;
            const K mk = ((K)((fams[f].ab >> 1) & 1u) << (q + n)) | ((K)(fams[f].ab & 1u) << q);
            entries.push_back(Entry{mk, 1u, (uint32_t)f | ((uint32_t)q << 16)});
        }
    }
    for (size_t g = 0; g < gens.size(); ++g) entries.push_back(Entry{gens[g].mask_key, 2u, (uint32_t)g});
    std::sort(entries.begin(), entries.end(),
              [](const Entry& a, const Entry& b) { return a.mask_key < b.mask_key; });

    // static weights per destination mask, from the expanded terms before
    // any merging (the proposal spawning's destination law)
    std::vector<StatSlot> stat;
    {
        // per mask, a saturating sum (order-free) over the sorted expanded terms
        int64_t run = 0;
        for (size_t a = 0, b = 0; a < sorted.size(); a = b) {
            const K mk = sorted[a].mk;
            int64_t acc = 0;
            for (b = a; b < sorted.size() && sorted[b].mk == mk; ++b) {
                const int64_t w = std::llabs(sorted[b].qre) + std::llabs(sorted[b].qim);
                acc = (acc >= (1ll << 52) || w >= (1ll << 52)) ? (1ll << 52) : std::min<int64_t>(acc + w, 1ll << 52);
            }
            if (acc == 0) continue;
            run = std::min<int64_t>(run + acc, 1ll << 52);
            stat.push_back(StatSlot{mk, run});
        }
        hdr.p_att = run;
    }

    // runs of consecutive members of one family (see Run)
    std::vector<Run> runs;
    for (size_t e = 0; e < entries.size(); ++e) {
        const Entry& E = entries[e];
        if (E.kind == 1u) {
            const uint32_t f = E.idx & 0xFFFFu, q = E.idx >> 16;
            if (!runs.empty() && runs.back().kind == 1u && runs.back().idx == f) {
                runs.back().members |= (M)1 << q;
                continue;
            }
            runs.push_back(Run{1u, f, (M)1 << q, (uint32_t)n});
        } else {
            runs.push_back(Run{E.kind, (uint32_t)e, (M)0, 0u});
        }
    }

    hdr.n_selffam = (int32_t)selffam.size();
    hdr.n_selfgen = (int32_t)selfgen.size();
    hdr.n_fam = (int32_t)fams.size();
    hdr.n_gen = (int32_t)gens.size();
    hdr.n_gterm = (int32_t)gterms.size();
    hdr.n_entry = (int32_t)entries.size();

    size_t base = align_up<A>(blob->size());
    size_t off = align_up<A>(sizeof(ProgHeader));
    hdr.off_selffam = (int32_t)off; off = align_up<A>(off + selffam.size() * sizeof(SelfFam));
    hdr.off_selfgen = (int32_t)off; off = align_up<A>(off + selfgen.size() * sizeof(SelfGen));
    hdr.off_fam = (int32_t)off;     off = align_up<A>(off + fams.size() * sizeof(Fam));
    hdr.off_gen = (int32_t)off;     off = align_up<A>(off + gens.size() * sizeof(Gen));
    hdr.off_gterm = (int32_t)off;   off = align_up<A>(off + gterms.size() * sizeof(GTerm));
    hdr.off_entry = (int32_t)off;   off = align_up<A>(off + entries.size() * sizeof(Entry));
    hdr.off_aff = (int32_t)off;     off = align_up<A>(off + affs.size() * sizeof(AffGroup));
    hdr.n_aff = (int32_t)affs.size();
    hdr.off_run = (int32_t)off;     off = align_up<A>(off + runs.size() * sizeof(Run));
    hdr.off_stat = (int32_t)off;    off = align_up<A>(off + stat.size() * sizeof(StatSlot));
    hdr.n_stat = (int32_t)stat.size();
    hdr.n_run = (int32_t)runs.size();
    hdr.bytes = (int32_t)off;
    blob->resize(base + off, 0);
    put(blob, base, &hdr, 1);
    put(blob, base + hdr.off_selffam, selffam.data(), selffam.size());
    put(blob, base + hdr.off_selfgen, selfgen.data(), selfgen.size());
    put(blob, base + hdr.off_fam, fams.data(), fams.size());
    put(blob, base + hdr.off_gen, gens.data(), gens.size());
    put(blob, base + hdr.off_gterm, gterms.data(), gterms.size());
    put(blob, base + hdr.off_entry, entries.data(), entries.size());
    put(blob, base + hdr.off_aff, affs.data(), affs.size());
    put(blob, base + hdr.off_run, runs.data(), runs.size());
    put(blob, base + hdr.off_stat, stat.data(), stat.size());
    return QMC_OK;
}

} // namespace

uint64_t schedule_hash(const Schedule& s, uint64_t seed, int32_t nseg, int32_t integrator,
                       int64_t n_diag, int64_t init_min)
{
    uint64_t h = 1469598103934665603ull;
    auto mix = [&](const void* p, size_t len) {
        const uint8_t* b = (const uint8_t*)p;
        for (size_t i = 0; i < len; ++i) { h ^= b[i]; h *= 1099511628211ull; }
    };
    mix(&s.n, sizeof(s.n));
    for (const auto& v : s.ham) { mix(&v.h, 8); mix(&v.xm, 8); mix(&v.zm, 8); mix(&v.rate_id, 4); mix(&v.window_id, 4); }
    for (const auto& v : s.lind) { mix(&v.first, 4); mix(&v.count, 4); mix(&v.rate_id, 4); mix(&v.window_id, 4); }
    for (const auto& v : s.coefs) { mix(&v.re, 8); mix(&v.im, 8); mix(&v.xm, 8); mix(&v.zm, 8); }
    for (const auto& v : s.rates) { mix(&v.kind, 4); mix(&v.a, 8); mix(&v.b, 8); mix(&v.c, 8); }
    for (const auto& v : s.windows) { mix(&v.t0, 8); mix(&v.t1, 8); }
    mix(&seed, 8); mix(&nseg, 4); mix(&integrator, 4); mix(&n_diag, 8); mix(&init_min, 8);
    return h;
}

} // namespace qmc
