// Library-internal data layouts shared by the host code and the kernels.
//
// Population record (16 B): one occupied state |x><y| of one vector,
//   key = (x << n) | y, value re + i im (int32 each) [walkers, Eq. (3)].
// Spawn record (16 B): key, meta, val.  meta = segment << 2 | target << 1 |
//   noninit, where target selects which component of the destination
//   receives val (0: re, 1: im) and noninit marks a spawn from a parent below
//   the initiator threshold [End Matter, simulation methodology].
//
// Key widths: up to 32 qubits a key is a uint64_t and a qubit mask a
// uint32_t; from 33 to 60 qubits a key is 128 bits (u128) and a mask a
// uint64_t (the "wide" layouts, records WRec / WSpawn, programs with the
// template arguments <uint64_t, u128>).
//
// Column program: the column of dt_eff * L(t) at |x><y| [Eq. (2)] for one step
// and one pass, in the 2^-52 fixed-point units of the expanded terms.  Terms
// are grouped by destination mask (dx << n | dy); a group's element is a sum
// of +-Q' over parity terms, the sign being the parity of popc(x & zl) +
// popc(y & zr).  Single-qubit groups that differ only by the qubit form a
// "family"; the per-qubit self (diagonal) parts form "self families".  Both
// are evaluated with popcounts, so the spawn probability of a parent costs a
// few integer operations regardless of n.
#pragma once
#include <stdint.h>

namespace qmc {

typedef unsigned __int128 u128;

struct Rec {
    uint64_t key;
    int32_t re, im;
};

struct SRec {
    uint64_t key;
    uint32_t meta;
    int32_t val;
};

static_assert(sizeof(Rec) == 16, "population record must be 16 bytes");
static_assert(sizeof(SRec) == 16, "spawn record must be 16 bytes");

// Wide records (33..60 qubits): the key (x << n) | y as two 64-bit words,
// compared high word first.  WRec is a record in registers; in memory a
// population slot stores its keys and its values as two arrays.
struct WRec {
    uint64_t lo, hi;
    int32_t re, im;
};

struct WSpawn {
    uint64_t lo, hi;
    uint32_t meta;   // segment << 2 | target << 1 | noninit, as in SRec
    int32_t val;
};

static_assert(sizeof(WRec) == 24, "wide population record must be 24 bytes");
static_assert(sizeof(WSpawn) == 24, "wide spawn record must be 24 bytes");

// ---- column program --------------------------------------------------------
struct ProgHeader {
    int32_t n_selffam, n_selfgen, n_fam, n_gen, n_gterm, n_entry;
    int32_t off_selffam, off_selfgen, off_fam, off_gen, off_gterm, off_entry;
    int32_t n_aff, off_aff;
    int32_t n_run, off_run;
    int32_t n_stat, off_stat;
    int64_t p_bound;                      // >= P of every state (filter for the spawn test)
    int64_t p_att;                        // proposal spawning: sum of the static weights (>= 2^52: too large)
    int64_t self_const_re, self_const_im; // parity-free part of the diagonal element
    int64_t p_const;                      // sum of |Re| + |Im| over constant groups
    int32_t bytes;                        // size of the whole blob
    int32_t n_nonconst_gen;               // generic groups come non-constant first
};

// Proposal spawning: every destination with a nonzero static weight (sum of
// |Re| + |Im| over its expanded terms), in ascending mask order, with the
// end of its interval in the cumulative static weights.
template <class K>
struct StatSlotT {
    K mask;
    int64_t end;
};

// Self-family parity term: Q' * (|M| - 2 popc(pat & M)), pat = x, y or x ^ y.
template <class M>
struct SelfFamT {
    M members;
    uint32_t type; // 0: zl = e_q (pattern x); 1: zr = e_q (y); 2: both (x ^ y)
    int64_t qre, qim;
};

// Self generic parity term (multi-qubit Z parity on the diagonal element).
template <class M>
struct SelfGenT {
    M zl, zr;
    int64_t qre, qim;
};

// Family of single-qubit groups: member q has destination mask
// (alpha e_q) << n | (beta e_q) and element tab[pi], pi = 2 x_q + y_q.
template <class M>
struct FamT {
    M members;
    uint32_t ab;   // bit 1: alpha (ket flips q), bit 0: beta (bra flips q)
    int64_t a[4];  // |Re tab| + |Im tab|
    int64_t tre[4], tim[4];
};

// Affine form of everything that depends on (x, y) only through the three
// counts cx = popc(x & M), cy = popc(y & M), c11 = popc(x & y & M) for one
// member mask M: the self-family part of the diagonal element,
//   s0 + sa cx + sb cy + sc c11   (complex),
// and the summed weight of the families with that mask,
//   f0 + fx cx + fy cy + f11 c11  (= sum over members of |Re T| + |Im T|).
template <class M>
struct AffGroupT {
    M members;
    uint32_t pad;
    int64_t s0re, s0im, sare, saim, sbre, sbim, scre, scim;
    int64_t f0, fx, fy, f11;
};

// Generic group: element = sum over terms [first, first + count) of +-Q'.
template <class K>
struct GenT {
    K mask_key;
    int32_t first, count;
    int32_t is_const, pad;
    int64_t cre, cim; // the element when is_const
};

template <class M>
struct GTermT {
    M zl, zr;
    int64_t qre, qim;
};

// Destinations of the column in ascending mask order (the canonical order of
// the multinomial choice).  kind 0: diagonal (mask 0); 1: family member
// (idx = fam | q << 16); 2: generic group (idx = gen).
template <class K>
struct EntryT {
    K mask_key;
    uint32_t kind;
    uint32_t idx;
};

// The entries as runs: a run of consecutive members of one family (ascending
// q, kind 1: idx = family, members = their q bits), or a single entry of
// kind 0 or 2 (idx = its entry index).  The destination choice walks runs and
// skips a family run by its summed weight.
template <class M>
struct RunT {
    uint32_t kind;
    uint32_t idx;
    M members;
    uint32_t shift;   // family runs: n (a member's ket bit is q + n)
};

// Narrow programs (up to 32 qubits).
using StatSlot = StatSlotT<uint64_t>;
using SelfFam = SelfFamT<uint32_t>;
using SelfGen = SelfGenT<uint32_t>;
using Fam = FamT<uint32_t>;
using AffGroup = AffGroupT<uint32_t>;
using Gen = GenT<uint64_t>;
using GTerm = GTermT<uint32_t>;
using Entry = EntryT<uint64_t>;
using Run = RunT<uint32_t>;

// ---- device-resident step state ---------------------------------------------
enum DevError : uint32_t {
    DERR_NONE = 0,
    DERR_SPAWN_CAPACITY = 1,
    DERR_POP_CAPACITY = 2,
    DERR_DT_TOO_LARGE = 3,
    DERR_POP_OVERFLOW = 4,
    DERR_TIMEOUT = 5,
    DERR_HEAVY_CAPACITY = 6,
    DERR_TILE_CAPACITY = 7,
    DERR_CAND_CAPACITY = 8,
    DERR_INTERNAL = 9,   // a step's self-check failed (counts of two kernels disagree)
};

constexpr int kMaxTileCounters = 32;

struct DevState {
    uint64_t step;        // global index of the next step
    int64_t count[3];     // records in population slots 0..2
    int32_t cur;          // slot of N(t); N(t - dt) is (cur + 2) % 3, output (cur + 1) % 3
    int32_t call_index;   // step index inside the current qmc_step call
    uint32_t error;       // sticky DevError
    uint32_t error_aux;
    int64_t spawn_total;  // spawn records requested this step
    int64_t heavy_total;  // heavy work items requested this step
    int64_t next_total;   // records produced by the merge this step
    int64_t merge_tiles;  // merge tiles this step
    int64_t cand_total;   // spawn candidates (draws below the bound) this step
    int64_t max_cand;
    int64_t max_spawn;    // high-water marks
    int64_t max_next;
    int64_t max_heavy;
    int64_t max_tiles;
    // cumulative counters since the last reset (qmc_counters)
    int64_t acc_steps;
    int64_t acc_walkers;  // sum over steps of N_tot of N(t + dt), all vectors
    int64_t acc_kcur;     // parents read from N(t)
    int64_t acc_kprev;    // parents read from N(t - dt) (AB2 steps)
    int64_t acc_spawn;    // spawn records written
    int64_t acc_knext;    // records written to N(t + dt)
    int64_t acc_heavy;    // heavy work items
    int64_t acc_cand;     // spawn candidates
    int64_t acc_sort_bucket;  // steps whose spawns took the bucket sort
    int64_t acc_sort_lsd;     // steps whose spawns took the LSD radix sort
    uint32_t seq;         // look-back epoch base, advanced by 16 every step
    uint32_t sort_fallback;   // 1: this step's spawns take the LSD radix sort
    uint32_t sort_final;      // 1: the sorted spawns end in the second spawn buffer
    uint32_t big_windows;     // buckets listed for the CTA sort
    uint32_t tile_ctr[kMaxTileCounters];
};

// Per-step flags prepared by the host for each step of a call.
struct StepInfo {
    int64_t tab_off;      // byte offset of int64[instances][2]: each instance's pass-0 / pass-1
                          // program offset (pass 1 repeats pass 0 when absent)
    int32_t ab2;          // 1: AB2 step (pass 1 over N(t - dt) present)
    int32_t pad;
    double t[2];          // time of pass 0 (t) and pass 1 (t - dt): input of the learned proposal
};

// Per population vector (segment): its problem instance, that instance's
// qubit count, and the vector's index inside the instance (which keys its
// random stream, so an instance run alone or in a batch draws the same).
struct SegInfo {
    int32_t inst;
    int32_t n;
    int32_t vec;
    int32_t pad;
};

// Per problem instance.
struct InstInfo {
    uint64_t seed;
    int64_t n_diag;
    int64_t init_min;   // initiator threshold in walkers (0: off)
    int32_t n;
    int32_t nvec;
};

} // namespace qmc
