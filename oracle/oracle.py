"""ctypes wrapper around the C oracle (test infrastructure only).

The oracle runs the plain method single-threaded: for every parent it builds
the Liouvillian column term by term [Eq. (1), Eq. (2)], draws one Philox word
per walker [End Matter, spawn step], and annihilates with a sorted merge
[End Matter, annihilation step].
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from .build import build

_lib = None

OK = 0
ERR_INVALID_ARG = -1
ERR_OOM = -2
ERR_DT_TOO_LARGE = -4
ERR_POP_OVERFLOW = -5
ERR_STATE = -8
ERR_COEF_RANGE = -9

EULER = 0
AB2 = 1


def _p(a, ctype):
    return a.ctypes.data_as(C.POINTER(ctype))


def lib():
    global _lib
    if _lib is None:
        path = build()
        L = C.CDLL(path)
        L.orc_problem_new.restype = C.c_void_p
        L.orc_problem_new.argtypes = [C.c_int] + [C.c_int, C.c_void_p, C.c_void_p, C.c_void_p,
                                                   C.c_void_p, C.c_void_p] + \
            [C.c_int, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p] + \
            [C.c_int, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p] + \
            [C.c_int, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p] + \
            [C.c_int, C.c_void_p, C.c_void_p]
        L.orc_problem_free.argtypes = [C.c_void_p]
        L.orc_column.restype = C.c_int
        L.orc_column.argtypes = [C.c_void_p, C.c_uint64, C.c_uint64, C.c_double, C.c_double,
                                 C.c_int, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]
        L.orc_static.restype = C.c_int
        L.orc_static.argtypes = [C.c_void_p, C.c_double, C.c_double, C.c_int, C.c_void_p, C.c_void_p,
                                 C.c_void_p]
        L.orc_state_new.restype = C.c_void_p
        L.orc_state_new.argtypes = [C.c_void_p, C.c_int, C.c_uint64, C.c_int, C.c_int64,
                                    C.c_int64]
        L.orc_state_free.argtypes = [C.c_void_p]
        L.orc_init.restype = C.c_int
        L.orc_init.argtypes = [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p,
                               C.c_void_p]
        L.orc_set_population_xy.restype = C.c_int
        L.orc_set_population_xy.argtypes = [C.c_void_p, C.c_int, C.c_int, C.c_int64] + [C.c_void_p] * 4
        L.orc_export_xy.restype = C.c_int
        L.orc_export_xy.argtypes = [C.c_void_p, C.c_int, C.c_int] + [C.c_void_p] * 4
        L.orc_next_value_xy.restype = C.c_int
        L.orc_next_value_xy.argtypes = [C.c_void_p, C.c_int, C.c_double, C.c_uint64, C.c_uint64, C.c_void_p]
        L.orc_set_population.restype = C.c_int
        L.orc_set_population.argtypes = [C.c_void_p, C.c_int, C.c_int, C.c_int64, C.c_void_p,
                                         C.c_void_p, C.c_void_p]
        L.orc_set_clock.restype = C.c_int
        L.orc_set_clock.argtypes = [C.c_void_p, C.c_uint64, C.c_double, C.c_double, C.c_double,
                                    C.c_int]
        L.orc_get_clock.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p]
        L.orc_set_active.restype = C.c_int
        L.orc_set_active.argtypes = [C.c_void_p, C.c_int, C.c_int]
        L.orc_set_proposal.restype = C.c_int
        L.orc_set_proposal.argtypes = [C.c_void_p, C.c_int]
        L.orc_set_mlp.restype = C.c_int
        L.orc_set_mlp.argtypes = [C.c_void_p, C.c_int, C.c_int, C.c_int] + [C.c_void_p] * 7 + [C.c_float]
        L.orc_step.restype = C.c_int
        L.orc_step.argtypes = [C.c_void_p, C.c_double, C.c_int]
        L.orc_count.restype = C.c_int64
        L.orc_count.argtypes = [C.c_void_p, C.c_int, C.c_int]
        L.orc_export.restype = C.c_int
        L.orc_export.argtypes = [C.c_void_p, C.c_int, C.c_int, C.c_void_p, C.c_void_p,
                                 C.c_void_p]
        L.orc_stats.argtypes = [C.c_void_p, C.c_int, C.c_void_p]
        L.orc_philox.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p]
        L.orc_zsum.argtypes = [C.c_void_p, C.c_int, C.c_void_p]
        L.orc_next_value.restype = C.c_int
        L.orc_next_value.argtypes = [C.c_void_p, C.c_int, C.c_double, C.c_uint64, C.c_void_p]
        L.orc_antiherm.argtypes = [C.c_void_p, C.c_int, C.c_void_p]
        L.orc_antiherm_sum.argtypes = [C.c_void_p, C.c_void_p, C.c_int, C.c_void_p]
        L.orc_walker_T.restype = C.c_int64
        L.orc_walker_T.argtypes = [C.c_void_p, C.c_int64, C.c_int, C.c_int, C.c_int64, C.c_int64]
        L.orc_mlp_exp.restype = C.c_float
        L.orc_mlp_exp.argtypes = [C.c_float]
        L.orc_learned_q.restype = C.c_int
        L.orc_learned_q.argtypes = [C.c_void_p, C.c_double, C.c_double, C.c_uint64, C.c_uint64, C.c_int,
                                    C.c_void_p, C.c_void_p, C.c_void_p]
        _lib = L
    return _lib


def walker_T(kd, rank: int, phase: int, comp: int, j: int, re_walkers: int) -> int:
    """The 52-bit spawn draw of walker j of component comp of the parent at
    `rank` in pass `phase` under the step key kd (two uint32)."""
    k = np.ascontiguousarray(kd, dtype=np.uint32)
    return int(lib().orc_walker_T(k.ctypes.data, rank, phase, comp, j, re_walkers))


def mlp_exp(x: float) -> float:
    """The learned proposal's single-precision e^x (x <= 0)."""
    return float(lib().orc_mlp_exp(float(x)))


def philox(ctr, key) -> np.ndarray:
    c = np.ascontiguousarray(np.asarray(ctr, dtype=np.uint32))
    k = np.ascontiguousarray(np.asarray(key, dtype=np.uint32))
    out = np.zeros(4, dtype=np.uint32)
    lib().orc_philox(c.ctypes.data, k.ctypes.data, out.ctypes.data)
    return out


class OracleProblem:
    """The oracle's own copy of a :class:`problems.Problem`."""

    def __init__(self, prob):
        self.prob = prob
        self.n = prob.n
        a = prob.arrays()
        self._keep = a
        L = lib()
        d = lambda k: a[k].ctypes.data if a[k].size else None  # noqa: E731
        self.handle = L.orc_problem_new(
            prob.n,
            len(a["h"]), d("h"), d("hx"), d("hz"), d("hrate"), d("hwin"),
            len(a["lstart"]), d("lstart"), d("lcount"), d("lrate"), d("lwin"),
            len(a["lre"]), d("lre"), d("lim"), d("lx"), d("lz"),
            len(a["rkind"]), d("rkind"), d("ra"), d("rb"), d("rc"),
            len(a["wt0"]), d("wt0"), d("wt1"))
        if not self.handle:
            raise ValueError("oracle rejected the problem")

    def _masks(self, lo, hi, k):
        """uint64 masks for n <= 32, else Python ints (dx << n | dy, 2n bits)."""
        if self.n <= 32:
            return lo[:k].copy()
        return np.array([(int(b) << 64) | int(a) for a, b in zip(lo[:k], hi[:k])], dtype=object)

    def column(self, x: int, y: int, t: float, dt_eff: float):
        """Quantised column of dt_eff * L(t) at |x><y|: (mask, qre, qim) sorted by mask,
        in units of 2^-52."""
        cap = 4096
        mask = np.zeros(cap, dtype=np.uint64)
        mask_hi = np.zeros(cap, dtype=np.uint64)
        qre = np.zeros(cap, dtype=np.int64)
        qim = np.zeros(cap, dtype=np.int64)
        n = lib().orc_column(self.handle, x, y, t, dt_eff, cap, mask.ctypes.data, mask_hi.ctypes.data,
                             qre.ctypes.data, qim.ctypes.data)
        if n < 0:
            raise RuntimeError(f"orc_column failed: {n}")
        return self._masks(mask, mask_hi, n), qre[:n].copy(), qim[:n].copy()

    def static(self, t: float, dt_eff: float):
        """Static weights of dt_eff * L(t): (mask, weight) sorted by mask, in
        units of 2^-52 (a bound on |Re L| + |Im L| of that destination)."""
        cap = 4096
        mask = np.zeros(cap, dtype=np.uint64)
        mask_hi = np.zeros(cap, dtype=np.uint64)
        w = np.zeros(cap, dtype=np.int64)
        n = lib().orc_static(self.handle, t, dt_eff, cap, mask.ctypes.data, mask_hi.ctypes.data, w.ctypes.data)
        if n < 0:
            raise RuntimeError(f"orc_static failed: {n}")
        return self._masks(mask, mask_hi, n), w[:n].copy()

    def __del__(self):
        if getattr(self, "handle", None):
            lib().orc_problem_free(self.handle)
            self.handle = None


class OracleSim:
    """Populations of ``nseg`` independent vectors evolved by the plain method."""

    def __init__(self, prob, nseg: int, seed: int, integrator: int = AB2,
                 init_min: int = 0, n_diag: int = 10000):
        self.problem = prob if isinstance(prob, OracleProblem) else OracleProblem(prob)
        self.n = self.problem.n
        self.nseg = nseg
        self.n_diag = n_diag
        self.handle = lib().orc_state_new(self.problem.handle, nseg, seed, integrator,
                                          init_min, n_diag)
        if not self.handle:
            raise ValueError("oracle rejected the state")

    def init(self, rho0):
        x = np.array([e[0] for e in rho0], dtype=np.uint64)
        y = np.array([e[1] for e in rho0], dtype=np.uint64)
        re = np.array([e[2] for e in rho0], dtype=np.float64)
        im = np.array([e[3] for e in rho0], dtype=np.float64)
        rc = lib().orc_init(self.handle, len(x), x.ctypes.data, y.ctypes.data, re.ctypes.data,
                            im.ctypes.data)
        if rc != OK:
            raise RuntimeError(f"orc_init failed: {rc}")

    def set_population(self, seg: int, keys, re, im, which: int = 0):
        keys = np.ascontiguousarray(keys, dtype=np.uint64)
        re = np.ascontiguousarray(re, dtype=np.int32)
        im = np.ascontiguousarray(im, dtype=np.int32)
        rc = lib().orc_set_population(self.handle, seg, which, len(keys), keys.ctypes.data,
                                      re.ctypes.data, im.ctypes.data)
        if rc != OK:
            raise RuntimeError(f"orc_set_population failed: {rc}")

    def set_population_xy(self, seg: int, x, y, re, im, which: int = 0):
        """Population of one vector from records |x><y| (any n)."""
        x = np.ascontiguousarray(x, dtype=np.uint64)
        y = np.ascontiguousarray(y, dtype=np.uint64)
        re = np.ascontiguousarray(re, dtype=np.int32)
        im = np.ascontiguousarray(im, dtype=np.int32)
        rc = lib().orc_set_population_xy(self.handle, seg, which, len(x), x.ctypes.data, y.ctypes.data,
                                         re.ctypes.data, im.ctypes.data)
        if rc != OK:
            raise RuntimeError(f"orc_set_population_xy failed: {rc}")

    def set_clock(self, step: int, t: float, t_prev: float = 0.0, dt_last: float = 0.0,
                  prev_valid: bool = False):
        lib().orc_set_clock(self.handle, step, t, t_prev, dt_last, int(prev_valid))

    def set_mlp(self, net):
        """Network of the learned proposal: a dict with out_masks (uint64), w1,
        b1, w2, b2, w3, b3 (float32, row-major) and eps."""
        arrs = [np.ascontiguousarray(net["out_masks"], dtype=np.uint64)] + \
            [np.ascontiguousarray(net[k], dtype=np.float32) for k in ("w1", "b1", "w2", "b2", "w3", "b3")]
        H, I = arrs[1].shape
        rc = lib().orc_set_mlp(self.handle, I, H, len(arrs[0]), *[a.ctypes.data for a in arrs],
                               float(net["eps"]))
        if rc != OK:
            raise RuntimeError(f"orc_set_mlp failed: {rc}")

    def learned_q(self, x: int, y: int, t: float, dt_eff: float):
        """The learned proposal's integer weights for the source |x><y|: (masks,
        Q, p_att) over the static column of dt_eff L(t) (after set_mlp)."""
        cap = 256
        mask = np.zeros(cap, dtype=np.uint64)
        Q = np.zeros(cap, dtype=np.int64)
        pa = np.zeros(1, dtype=np.int64)
        k = lib().orc_learned_q(self.handle, t, dt_eff, x, y, cap, mask.ctypes.data, Q.ctypes.data,
                                pa.ctypes.data)
        if k < 0:
            raise RuntimeError(f"orc_learned_q failed: {k}")
        return mask[:k], Q[:k], int(pa[0])

    def set_proposal(self, kind: int):
        """Spawn choice: 0 exact |L|-weighted (the paper's), 1 static-weight
        proposal, 2 learned proposal (after set_mlp)."""
        rc = lib().orc_set_proposal(self.handle, kind)
        if rc != OK:
            raise RuntimeError(f"orc_set_proposal failed: {rc}")

    def set_active(self, segs):
        """Step only the listed vectors (the others keep their populations)."""
        segs = set(segs)
        for s in range(self.nseg):
            lib().orc_set_active(self.handle, s, 1 if s in segs else 0)

    def clock(self):
        step = np.zeros(1, dtype=np.uint64)
        tt = np.zeros(4, dtype=np.float64)
        lib().orc_get_clock(self.handle, step.ctypes.data, tt.ctypes.data)
        return int(step[0]), float(tt[0]), float(tt[1]), float(tt[2]), bool(tt[3])

    def step(self, dt: float, nsteps: int = 1) -> int:
        return lib().orc_step(self.handle, dt, nsteps)

    def population(self, seg: int, which: int = 0):
        cnt = lib().orc_count(self.handle, seg, which)
        keys = np.zeros(cnt, dtype=np.uint64)
        re = np.zeros(cnt, dtype=np.int32)
        im = np.zeros(cnt, dtype=np.int32)
        if cnt:
            lib().orc_export(self.handle, seg, which, keys.ctypes.data, re.ctypes.data,
                             im.ctypes.data)
        return keys, re, im

    def population_xy(self, seg: int, which: int = 0):
        """One vector's population as (x, y, re, im) in key order (any n)."""
        cnt = lib().orc_count(self.handle, seg, which)
        x = np.zeros(cnt, dtype=np.uint64)
        y = np.zeros(cnt, dtype=np.uint64)
        re = np.zeros(cnt, dtype=np.int32)
        im = np.zeros(cnt, dtype=np.int32)
        if cnt:
            lib().orc_export_xy(self.handle, seg, which, x.ctypes.data, y.ctypes.data, re.ctypes.data,
                                im.ctypes.data)
        return x, y, re, im

    def next_value_xy(self, seg: int, dt: float, x: int, y: int):
        """next_value at the state |x><y| (any n)."""
        out = np.zeros(2, dtype=np.int64)
        rc = lib().orc_next_value_xy(self.handle, seg, dt, x, y, out.ctypes.data)
        if rc != OK:
            raise RuntimeError(f"orc_next_value_xy failed: {rc}")
        return int(out[0]), int(out[1])

    def next_value(self, seg: int, dt: float, key: int):
        """(re, im) that the next step of size dt leaves at `key` of vector
        seg, computed from the parents that can reach it (no step taken)."""
        out = np.zeros(2, dtype=np.int64)
        rc = lib().orc_next_value(self.handle, seg, dt, key, out.ctypes.data)
        if rc != OK:
            raise RuntimeError(f"orc_next_value failed: {rc}")
        return int(out[0]), int(out[1])

    def zsum(self, seg: int) -> np.ndarray:
        """Per qubit q: sum over diagonal records of Re N_xx (-1)^(x_q)."""
        out = np.zeros(self.n, dtype=np.int64)
        lib().orc_zsum(self.handle, seg, out.ctypes.data)
        return out

    def antiherm(self, seg: int) -> int:
        """||N - N^dagger||_F^2 of one vector, an exact integer."""
        out = np.zeros(2, dtype=np.uint64)
        lib().orc_antiherm(self.handle, seg, out.ctypes.data)
        return int(out[0]) + (int(out[1]) << 64)

    def antiherm_sum(self, segs) -> int:
        """||S - S^dagger||_F^2 of the sum S of the listed vectors, exact."""
        sg = np.ascontiguousarray(segs, dtype=np.int32)
        out = np.zeros(2, dtype=np.uint64)
        lib().orc_antiherm_sum(self.handle, sg.ctypes.data, len(sg), out.ctypes.data)
        return int(out[0]) + (int(out[1]) << 64)

    def stats(self, seg: int):
        out = np.zeros(4, dtype=np.int64)
        lib().orc_stats(self.handle, seg, out.ctypes.data)
        return out

    def density(self, seg: int) -> np.ndarray:
        """Dense N(t) of one vector as a D x D complex matrix (tiny n only)."""
        D = 1 << self.n
        rho = np.zeros((D, D), dtype=np.complex128)
        keys, re, im = self.population(seg)
        x = (keys >> np.uint64(self.n)).astype(np.int64)
        y = (keys & np.uint64(D - 1)).astype(np.int64)
        rho[x, y] = re + 1j * im
        return rho

    def __del__(self):
        if getattr(self, "handle", None):
            lib().orc_state_free(self.handle)
            self.handle = None
