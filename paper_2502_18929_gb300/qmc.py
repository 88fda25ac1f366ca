"""ctypes binding of ``libqmc_gb300.so`` (include/qmc.h): argument marshalling only.

Every step of the method runs in the library's CUDA kernels; this module
converts NumPy / torch arguments to the C structs and back.  There is no CPU
fallback: importing works without a GPU, but creating a context fails loudly
if the library or a CUDA device is missing.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

OK = 0
ERR_INVALID_ARG = -1
ERR_OOM = -2
ERR_CAPACITY = -3
ERR_DT_TOO_LARGE = -4
ERR_POP_OVERFLOW = -5
ERR_DEVICE_TIMEOUT = -6
ERR_CUDA = -7
ERR_STATE = -8
ERR_COEF_RANGE = -9
ERR_IO = -10
ERR_CHECKPOINT = -11

EULER = 0
AB2 = 1
PROPOSAL_EXACT, PROPOSAL_STATIC, PROPOSAL_LEARNED, PROPOSAL_LEARNED_TC = 0, 1, 2, 3

EXPORTED = [
    "qmc_create", "qmc_destroy", "qmc_last_error", "qmc_load_schedule", "qmc_init_populations",
    "qmc_set_populations", "qmc_set_clock", "qmc_get_clock", "qmc_step", "qmc_spawn_prob_bound",
    "qmc_observables", "qmc_step_history", "qmc_export", "qmc_overlap", "qmc_checkpoint", "qmc_restore",
    "qmc_step_profile", "qmc_kernel_name", "qmc_column_eval", "qmc_counters", "qmc_observables_noalloc",
    "qmc_step_launches", "qmc_batch_create", "qmc_set_proposal", "qmc_set_proposal_mlp",
    "qmc_learn_param_count", "qmc_learn_events", "qmc_learn_grad", "qmc_learn_adam", "qmc_learn_load",
    "qmc_set_tuning", "qmc_get_tuning", "qmc_autotune", "qmc_set_spin_limit", "qmc_z_history",
    "qmc_overlap_all", "qmc_antihermiticity", "qmc_antihermiticity_sum", "qmc_learn_grad_tc", "qmc_memory",
    "qmc_export_xy", "qmc_set_populations_xy", "qmc_step_kernel_name", "qmc_learned_weights",
]


class QmcError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{msg} (code {code})")
        self.code = code


ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_uint64, C.c_void_p, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p, C.c_void_p)


class Config(C.Structure):
    _fields_ = [("n_qubits", C.c_int32), ("n_segments", C.c_int32), ("integrator", C.c_int32),
                ("max_ctas", C.c_int32), ("seed", C.c_uint64), ("n_diag", C.c_int64),
                ("initiator_min", C.c_int64), ("capacity_hint", C.c_int64), ("max_records", C.c_int64),
                ("cuda_stream", C.c_void_p), ("alloc", ALLOC_FN), ("free", FREE_FN), ("alloc_user", C.c_void_p)]


class TorchAllocator:
    """Device memory of a context from torch's caching allocator (the
    qmc_config.alloc / free callbacks): blocks are taken and returned in
    stream order on the context's work stream.  ``calls`` counts
    [allocations, frees]."""

    def __init__(self, device: int | None = None):
        import torch
        self.device = torch.cuda.current_device() if device is None else int(device)
        self.calls = [0, 0]

        def _alloc(nbytes, stream, user):
            try:
                p = torch.cuda.caching_allocator_alloc(int(nbytes), self.device, int(stream or 0))
                self.calls[0] += 1
                return p
            except Exception:   # out of memory: the library reports QMC_ERR_OOM
                return None

        def _free(ptr, stream, user):
            self.calls[1] += 1
            torch.cuda.caching_allocator_delete(ptr)

        self.alloc = ALLOC_FN(_alloc)
        self.free = FREE_FN(_free)

    def attach(self, cfg: Config):
        cfg.alloc = self.alloc
        cfg.free = self.free


class HamTerm(C.Structure):
    _fields_ = [("h", C.c_double), ("xm", C.c_uint64), ("zm", C.c_uint64), ("rate_id", C.c_int32),
                ("window_id", C.c_int32)]


class PauliCoef(C.Structure):
    _fields_ = [("re", C.c_double), ("im", C.c_double), ("xm", C.c_uint64), ("zm", C.c_uint64)]


class Lindblad(C.Structure):
    _fields_ = [("first", C.c_int32), ("count", C.c_int32), ("rate_id", C.c_int32), ("window_id", C.c_int32)]


class Rate(C.Structure):
    _fields_ = [("kind", C.c_int32), ("pad", C.c_int32), ("a", C.c_double), ("b", C.c_double),
                ("c", C.c_double)]


class Window(C.Structure):
    _fields_ = [("t0", C.c_double), ("t1", C.c_double)]


class Obs(C.Structure):
    _fields_ = [("n_records", C.c_int64), ("n_walkers", C.c_int64), ("n_diag_re", C.c_int64),
                ("n_diag_im", C.c_int64)]


_lib = None


def library_path() -> str:
    return _build.LIB


def lib():
    """Load (building first if needed) the CUDA library."""
    global _lib
    if _lib is None:
        path = _build.LIB
        if not os.path.exists(path):
            path = _build.build()
        L = C.CDLL(path)
        vp = C.c_void_p
        L.qmc_create.argtypes = [C.POINTER(vp), C.POINTER(Config)]
        L.qmc_destroy.argtypes = [vp]
        L.qmc_destroy.restype = None
        L.qmc_last_error.argtypes = [vp]
        L.qmc_last_error.restype = C.c_char_p
        L.qmc_load_schedule.argtypes = [vp, vp, C.c_int32, vp, C.c_int32, vp, C.c_int32, vp, C.c_int32, vp,
                                        C.c_int32]
        L.qmc_init_populations.argtypes = [vp, vp, vp, vp, vp, C.c_int64]
        L.qmc_set_populations.argtypes = [vp, C.c_int32, vp, vp, vp, vp]
        L.qmc_set_clock.argtypes = [vp, C.c_uint64, C.c_double, C.c_double, C.c_double, C.c_int32]
        L.qmc_get_clock.argtypes = [vp, vp, vp, vp, vp, vp]
        L.qmc_step.argtypes = [vp, C.c_double, C.c_int64]
        L.qmc_spawn_prob_bound.argtypes = [vp, C.c_double, C.c_double, vp]
        L.qmc_observables.argtypes = [vp, vp]
        L.qmc_step_history.argtypes = [vp, vp, C.c_int64, vp]
        L.qmc_export.argtypes = [vp, C.c_int32, C.c_int32, vp, vp, vp, C.c_int64, vp]
        L.qmc_overlap.argtypes = [vp, C.c_int32, vp, vp, vp, C.c_int32, vp, vp]
        L.qmc_checkpoint.argtypes = [vp, C.c_char_p]
        L.qmc_restore.argtypes = [vp, C.c_char_p]
        L.qmc_step_profile.argtypes = [vp, C.c_double, C.c_int64, vp, C.c_int32, vp]
        L.qmc_counters.argtypes = [vp, C.c_int32, vp]
        L.qmc_step_launches.argtypes = [vp, vp]
        L.qmc_set_proposal.argtypes = [vp, C.c_int32]
        L.qmc_set_proposal_mlp.argtypes = [vp, C.POINTER(Mlp)]
        L.qmc_learn_param_count.argtypes = [vp, vp]
        L.qmc_learn_events.argtypes = [vp, C.c_double, C.c_int64, vp, vp, vp, vp]
        L.qmc_learn_grad.argtypes = [vp, vp, vp, vp, vp, C.c_int64, C.c_int64, vp, vp]
        L.qmc_learn_grad_tc.argtypes = [vp, vp, vp, vp, vp, C.c_int64, C.c_int64, vp, vp]
        L.qmc_learn_adam.argtypes = [vp, vp, vp, vp, vp, C.c_int64, C.c_int64, C.c_float, C.c_float, C.c_float,
                                     C.c_float]
        L.qmc_learn_load.argtypes = [vp, vp]
        L.qmc_set_tuning.argtypes = [vp, C.POINTER(Tuning)]
        L.qmc_get_tuning.argtypes = [vp, C.POINTER(Tuning)]
        L.qmc_autotune.argtypes = [vp, C.c_double, C.c_int32, C.POINTER(Tuning)]
        L.qmc_set_spin_limit.argtypes = [vp, C.c_uint32]
        L.qmc_z_history.argtypes = [vp, vp, C.c_int64, vp]
        L.qmc_overlap_all.argtypes = [vp, vp, vp, vp, C.c_int32, vp, vp]
        L.qmc_antihermiticity.argtypes = [vp, vp]
        L.qmc_antihermiticity_sum.argtypes = [vp, vp, C.c_int32, vp]
        L.qmc_batch_create.argtypes = [C.POINTER(vp), vp, C.c_int32, C.POINTER(Config)]
        L.qmc_observables_noalloc.argtypes = [vp, vp, C.c_int32, C.c_int32, vp, vp]
        L.qmc_memory.argtypes = [vp, vp]
        L.qmc_set_populations_xy.argtypes = [vp, C.c_int32, vp, vp, vp, vp, vp]
        L.qmc_learned_weights.argtypes = [vp, C.c_double, C.c_double, vp, vp, C.c_int32, vp, C.c_int32,
                                          C.POINTER(C.c_int32)]
        L.qmc_export_xy.argtypes = [vp, C.c_int32, C.c_int32, vp, vp, vp, vp, C.c_int64, C.POINTER(C.c_int64)]
        L.qmc_kernel_name.argtypes = [C.c_int32]
        L.qmc_kernel_name.restype = C.c_char_p
        L.qmc_step_kernel_name.argtypes = [vp, C.c_int32]
        L.qmc_step_kernel_name.restype = C.c_char_p
        for name in EXPORTED:
            if name not in ("qmc_destroy", "qmc_last_error", "qmc_kernel_name", "qmc_step_kernel_name",
                            "qmc_column_eval"):
                getattr(L, name).restype = C.c_int
        _lib = L
    return _lib


def _arr(a, dtype):
    return np.ascontiguousarray(np.asarray(a, dtype=dtype))


def _ptr(a):
    return a.ctypes.data if a.size else None


def current_stream_handle() -> int:
    """The torch current CUDA stream (0 = legacy default stream)."""
    try:
        import torch
        if torch.cuda.is_available() and torch.cuda.is_initialized():
            return int(torch.cuda.current_stream().cuda_stream)
    except Exception:
        pass
    return 0


class Tuning(C.Structure):
    _fields_ = [("max_ctas", C.c_int32), ("heavy_walkers", C.c_int32), ("bucket_records", C.c_int32),
                ("pad", C.c_int32)]


class Mlp(C.Structure):
    _fields_ = [("n_in", C.c_int32), ("n_hidden", C.c_int32), ("n_out", C.c_int32), ("eps", C.c_float),
                ("out_masks", C.c_void_p), ("w1", C.c_void_p), ("b1", C.c_void_p), ("w2", C.c_void_p),
                ("b2", C.c_void_p), ("w3", C.c_void_p), ("b3", C.c_void_p)]


class Instance(C.Structure):
    _fields_ = [("n_qubits", C.c_int32), ("n_vectors", C.c_int32), ("seed", C.c_uint64), ("n_diag", C.c_int64),
                ("initiator_min", C.c_int64), ("ham", C.c_void_p), ("n_ham", C.c_int32), ("n_lind", C.c_int32),
                ("lind", C.c_void_p), ("coefs", C.c_void_p), ("n_coefs", C.c_int32), ("n_rates", C.c_int32),
                ("rates", C.c_void_p), ("windows", C.c_void_p), ("n_windows", C.c_int32), ("pad", C.c_int32)]


def _schedule_arrays(prob):
    """ctypes arrays of a problem's schedule (kept alive by the caller)."""
    ham = (HamTerm * max(1, len(prob.ham)))(*[HamTerm(h, xm, zm, r, w) for h, xm, zm, r, w in prob.ham])
    coefs, linds = [], []
    for ops, r, w in prob.lind:
        linds.append(Lindblad(len(coefs), len(ops), r, w))
        for coef, xm, zm in ops:
            coefs.append(PauliCoef(coef.real, coef.imag, xm, zm))
    lind = (Lindblad * max(1, len(linds)))(*linds)
    cf = (PauliCoef * max(1, len(coefs)))(*coefs)
    rates = (Rate * max(1, len(prob.rates)))(*[Rate(k, 0, a, b, c) for k, a, b, c in prob.rates])
    wins = (Window * max(1, len(prob.windows)))(*[Window(a, b) for a, b in prob.windows])
    return ham, len(prob.ham), lind, len(linds), cf, len(coefs), rates, len(prob.rates), wins, len(prob.windows)


class QMC:
    """One context: ``n_segments`` independent population vectors of one problem."""

    def __init__(self, n_qubits: int, n_segments: int, seed: int, n_diag: int, integrator: int = AB2,
                 initiator_min: int = 0, capacity_hint: int = 0, max_records: int = 0, stream: int | None = None,
                 max_ctas: int = 0, allocator: "TorchAllocator | None" = None):
        self.L = lib()
        self.n = n_qubits
        self.nseg = n_segments
        self.n_diag = n_diag
        cfg = Config(n_qubits, n_segments, integrator, max_ctas, seed, n_diag, initiator_min, capacity_hint,
                     max_records, C.c_void_p(current_stream_handle() if stream is None else stream))
        self._allocator = allocator   # its callbacks must outlive the context
        if allocator is not None:
            allocator.attach(cfg)
        h = C.c_void_p()
        rc = self.L.qmc_create(C.byref(h), C.byref(cfg))
        if rc != OK:
            raise QmcError(rc, "qmc_create failed (is a CUDA device present?)")
        self.h = h

    def _check(self, rc: int, what: str):
        if rc != OK:
            raise QmcError(rc, f"{what}: {self.L.qmc_last_error(self.h).decode()}")

    def close(self):
        if getattr(self, "h", None):
            self.L.qmc_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- problem -------------------------------------------------------------
    @classmethod
    def batch(cls, problems, n_vectors, seeds, n_diags, integrator: int = AB2, initiator_mins=None,
              capacity_hint: int = 0, max_records: int = 0, stream: int | None = None, max_ctas: int = 0,
              allocator: "TorchAllocator | None" = None):
        """One context stepping several problem instances (qmc_batch_create):
        instance i's vectors are segments offsets[i] .. offsets[i + 1]."""
        self = cls.__new__(cls)
        self.L = lib()
        self._allocator = allocator
        k = len(problems)
        mins = initiator_mins if initiator_mins is not None else [0] * k
        keep, arr = [], (Instance * k)()
        for i, prob in enumerate(problems):
            a = _schedule_arrays(prob)
            keep.append(a)
            ham, nh, lind, nl, cf, nc, rates, nr, wins, nw = a
            arr[i] = Instance(prob.n, int(n_vectors[i]), int(seeds[i]), int(n_diags[i]), int(mins[i]),
                              C.cast(ham, C.c_void_p), nh, nl, C.cast(lind, C.c_void_p), C.cast(cf, C.c_void_p),
                              nc, nr, C.cast(rates, C.c_void_p), C.cast(wins, C.c_void_p), nw, 0)
        cfg = Config(max(p.n for p in problems), int(sum(n_vectors)), integrator, max_ctas, 0, 1, 0, capacity_hint,
                     max_records, C.c_void_p(current_stream_handle() if stream is None else stream))
        if allocator is not None:
            allocator.attach(cfg)
        h = C.c_void_p()
        rc = self.L.qmc_batch_create(C.byref(h), arr, k, C.byref(cfg))
        if rc != OK:
            raise QmcError(rc, "qmc_batch_create failed")
        self.h = h
        self.n = cfg.n_qubits
        self.nseg = cfg.n_segments
        self.n_diag = None
        self.offsets = np.concatenate([[0], np.cumsum(n_vectors)]).astype(np.int64)
        return self

    def set_proposal(self, kind: int):
        """Spawn choice: EXACT (0, the paper's), STATIC (1, static-weight
        proposal) or LEARNED (2, after set_mlp)."""
        self._check(self.L.qmc_set_proposal(self.h, kind), "qmc_set_proposal")

    def set_mlp(self, net):
        """Network of the learned proposal: a dict with out_masks (uint64), w1,
        b1, w2, b2, w3, b3 (float32, row-major) and eps."""
        arrs = [np.ascontiguousarray(net["out_masks"], dtype=np.uint64)] + \
            [np.ascontiguousarray(net[k], dtype=np.float32) for k in ("w1", "b1", "w2", "b2", "w3", "b3")]
        H, I = arrs[1].shape
        m = Mlp(I, H, len(arrs[0]), float(net["eps"]), *[a.ctypes.data for a in arrs])
        self._check(self.L.qmc_set_proposal_mlp(self.h, C.byref(m)), "qmc_set_proposal_mlp")
        self._mlp_out = len(arrs[0])

    # -- launch shapes ----------------------------------------------------------
    def set_tuning(self, max_ctas: int = 0, heavy_walkers: int = 256, bucket_records: int = 24):
        t = Tuning(max_ctas, heavy_walkers, bucket_records, 0)
        self._check(self.L.qmc_set_tuning(self.h, C.byref(t)), "qmc_set_tuning")

    def set_spin_limit(self, polls: int = 1 << 22):
        """Polls of another CTA's look-back word before a device wait gives up
        (the step then fails with ERR_DEVICE_TIMEOUT); 0 fails every such wait."""
        self._check(self.L.qmc_set_spin_limit(self.h, polls), "qmc_set_spin_limit")

    def get_tuning(self) -> dict:
        t = Tuning()
        self._check(self.L.qmc_get_tuning(self.h, C.byref(t)), "qmc_get_tuning")
        return {"max_ctas": t.max_ctas, "heavy_walkers": t.heavy_walkers, "bucket_records": t.bucket_records}

    def autotune(self, dt: float, nsteps: int = 4) -> dict:
        """Time candidate launch shapes from the current state (which is kept)
        and leave the fastest set; returns them."""
        t = Tuning()
        self._check(self.L.qmc_autotune(self.h, dt, nsteps, C.byref(t)), "qmc_autotune")
        return {"max_ctas": t.max_ctas, "heavy_walkers": t.heavy_walkers, "bucket_records": t.bucket_records}

    # -- training of the learned proposal (device tensors) ---------------------
    def learned_weights(self, t: float, dt_eff: float, xs, ys, cap_slots: int = 256) -> np.ndarray:
        """The learned proposal's integer weights (count, n_slots) for sources
        |x><y| under the static column of dt_eff L(t) (qmc_learned_weights)."""
        x, y = _arr(xs, np.uint64), _arr(ys, np.uint64)
        Q = np.zeros((max(1, len(x)), cap_slots), dtype=np.int64)
        ns = C.c_int32()
        self._check(self.L.qmc_learned_weights(self.h, t, dt_eff, _ptr(x), _ptr(y), len(x), Q.ctypes.data, cap_slots,
                                               C.byref(ns)), "qmc_learned_weights")
        return Q[:len(x), :ns.value]

    def learn_param_count(self) -> int:
        n = C.c_int64()
        self._check(self.L.qmc_learn_param_count(self.h, C.byref(n)), "qmc_learn_param_count")
        return n.value

    def learn_events(self, dt: float, max_events: int):
        """Events from N(t): (feat [2n+1, max_events], target [G, max_events],
        weight [max_events]) float32 CUDA tensors and the event count."""
        import torch
        G = getattr(self, "_mlp_out", 1)   # without a network the library reports the error
        feat = torch.empty((2 * self.n + 1, max_events), dtype=torch.float32, device="cuda")
        target = torch.empty((G, max_events), dtype=torch.float32, device="cuda")
        weight = torch.empty(max_events, dtype=torch.float32, device="cuda")
        ne = C.c_int64()
        self._check(self.L.qmc_learn_events(self.h, dt, max_events, feat.data_ptr(), target.data_ptr(),
                                            weight.data_ptr(), C.byref(ne)), "qmc_learn_events")
        return feat, target, weight, ne.value

    def learn_grad(self, params, feat, target, weight, n_events: int):
        """(loss, grad) of the packed parameters over the first n_events events."""
        import torch
        grad = torch.empty_like(params)
        loss = C.c_double()
        self._check(self.L.qmc_learn_grad(self.h, params.data_ptr(), feat.data_ptr(), target.data_ptr(),
                                          weight.data_ptr(), feat.shape[1], n_events, grad.data_ptr(),
                                          C.byref(loss)), "qmc_learn_grad")
        return loss.value, grad

    def learn_grad_tc(self, params, feat, target, weight, n_events: int):
        """(loss, grad) of the tensor-core network (bf16, GELU) over the first
        n_events events."""
        import torch
        grad = torch.empty_like(params)
        loss = C.c_double()
        self._check(self.L.qmc_learn_grad_tc(self.h, params.data_ptr(), feat.data_ptr(), target.data_ptr(),
                                             weight.data_ptr(), feat.shape[1], n_events, grad.data_ptr(),
                                             C.byref(loss)), "qmc_learn_grad_tc")
        return loss.value, grad

    def learn_adam(self, params, grad, m, v, t: int, lr: float, beta1: float = 0.9, beta2: float = 0.999,
                   eps: float = 1e-8):
        self._check(self.L.qmc_learn_adam(self.h, params.data_ptr(), grad.data_ptr(), m.data_ptr(), v.data_ptr(),
                                          params.numel(), t, lr, beta1, beta2, eps), "qmc_learn_adam")

    def learn_load(self, params):
        self._check(self.L.qmc_learn_load(self.h, params.data_ptr()), "qmc_learn_load")

    def load_schedule(self, prob):
        a = _schedule_arrays(prob)
        self._check(self.L.qmc_load_schedule(self.h, *a), "qmc_load_schedule")

    def init_populations(self, rho0):
        x = _arr([e[0] for e in rho0], np.uint64)
        y = _arr([e[1] for e in rho0], np.uint64)
        re = _arr([e[2] for e in rho0], np.float64)
        im = _arr([e[3] for e in rho0], np.float64)
        self._check(self.L.qmc_init_populations(self.h, _ptr(x), _ptr(y), _ptr(re), _ptr(im), len(x)),
                    "qmc_init_populations")

    def set_populations(self, pops, which: int = 0):
        """``pops``: list (one per vector) of (keys ascending, re, im)."""
        counts = _arr([len(p[0]) for p in pops], np.int64)
        keys = _arr(np.concatenate([np.asarray(p[0], dtype=np.uint64) for p in pops]), np.uint64)
        re = _arr(np.concatenate([np.asarray(p[1], dtype=np.int32) for p in pops]), np.int32)
        im = _arr(np.concatenate([np.asarray(p[2], dtype=np.int32) for p in pops]), np.int32)
        self._check(self.L.qmc_set_populations(self.h, which, _ptr(counts), _ptr(keys), _ptr(re), _ptr(im)),
                    "qmc_set_populations")

    def set_populations_packed(self, counts, keys, re, im, which: int = 0):
        """As set_populations, from back-to-back arrays (any host memory; pinned
        memory uploads at full link speed)."""
        counts = _arr(counts, np.int64)
        for a, dt in ((keys, np.uint64), (re, np.int32), (im, np.int32)):
            if a.dtype != dt or not a.flags["C_CONTIGUOUS"]:
                raise TypeError("keys must be C-contiguous uint64 and re/im int32")
        self._check(self.L.qmc_set_populations(self.h, which, _ptr(counts), _ptr(keys), _ptr(re), _ptr(im)),
                    "qmc_set_populations")

    def set_populations_xy(self, counts, x, y, re, im, which: int = 0):
        """Populations from concatenated per-vector records |x><y| (any n),
        (x, y) ascending within each vector."""
        counts = _arr(counts, np.int64)
        x, y = _arr(x, np.uint64), _arr(y, np.uint64)
        re, im = _arr(re, np.int32), _arr(im, np.int32)
        self._check(self.L.qmc_set_populations_xy(self.h, which, counts.ctypes.data, _ptr(x), _ptr(y), _ptr(re),
                                                  _ptr(im)), "qmc_set_populations_xy")

    def set_clock(self, step: int, t: float, t_prev: float = 0.0, dt_last: float = 0.0,
                  prev_valid: bool = False):
        self._check(self.L.qmc_set_clock(self.h, step, t, t_prev, dt_last, int(prev_valid)), "qmc_set_clock")

    def clock(self):
        step = C.c_uint64()
        t, tp, dl = C.c_double(), C.c_double(), C.c_double()
        pv = C.c_int32()
        self._check(self.L.qmc_get_clock(self.h, C.byref(step), C.byref(t), C.byref(tp), C.byref(dl),
                                         C.byref(pv)), "qmc_get_clock")
        return step.value, t.value, tp.value, dl.value, bool(pv.value)

    def set_time(self, t: float):
        step, _, tp, dl, pv = self.clock()
        self.set_clock(step, t, tp, dl, pv)

    # -- hot path --------------------------------------------------------------
    def step(self, dt: float, nsteps: int = 1):
        self._check(self.L.qmc_step(self.h, dt, nsteps), "qmc_step")

    def step_rc(self, dt: float, nsteps: int = 1) -> int:
        return self.L.qmc_step(self.h, dt, nsteps)

    def step_profile(self, dt: float, nsteps: int = 1) -> dict:
        """Per-kernel milliseconds summed over nsteps steps (CUDA events)."""
        ms = np.zeros(32, dtype=np.float64)
        nk = C.c_int32()
        self._check(self.L.qmc_step_profile(self.h, dt, nsteps, ms.ctypes.data, 32, C.byref(nk)),
                    "qmc_step_profile")
        return {self.L.qmc_step_kernel_name(self.h, i).decode(): float(ms[i]) for i in range(nk.value)}

    def memory(self) -> dict:
        """Device memory the context holds (qmc_memory)."""
        out = np.zeros(2, dtype=np.int64)
        self._check(self.L.qmc_memory(self.h, out.ctypes.data), "qmc_memory")
        return {"bytes": int(out[0]), "blocks": int(out[1])}

    def counters(self, reset: bool = False) -> dict:
        """Cumulative device totals since the last reset (see qmc_counters)."""
        out = np.zeros(11, dtype=np.int64)
        self._check(self.L.qmc_counters(self.h, int(reset), out.ctypes.data), "qmc_counters")
        names = ["steps", "walker_steps", "k_cur", "k_prev", "spawns", "k_next", "heavy_items", "candidates",
                 "sort_bucket_steps", "sort_lsd_steps", "redo_launches"]
        return {k: int(v) for k, v in zip(names, out)}

    def step_launches(self) -> int:
        """Kernel launches of one step as the context would issue it now."""
        n = C.c_int32()
        self._check(self.L.qmc_step_launches(self.h, C.byref(n)), "qmc_step_launches")
        return n.value

    def spawn_prob_bound(self, t: float, dt: float) -> float:
        p = C.c_double()
        self._check(self.L.qmc_spawn_prob_bound(self.h, t, dt, C.byref(p)), "qmc_spawn_prob_bound")
        return p.value

    # -- results --------------------------------------------------------------
    def observables(self) -> np.ndarray:
        """(n_segments, 4) int64: K, N_tot, Re N^diag, Im N^diag."""
        out = np.zeros((self.nseg, 4), dtype=np.int64)
        self._check(self.L.qmc_observables(self.h, out.ctypes.data), "qmc_observables")
        return out

    def step_history(self, cap_steps: int = 1 << 20) -> np.ndarray:
        """(steps, n_segments, 4) int64 for every step of the last ``step`` call."""
        _, _, _, _, _ = self.clock()
        buf = np.zeros((max(1, min(cap_steps, 1 << 22)), self.nseg, 4), dtype=np.int64)
        cnt = C.c_int64()
        self._check(self.L.qmc_step_history(self.h, buf.ctypes.data, buf.shape[0], C.byref(cnt)),
                    "qmc_step_history")
        return buf[:cnt.value]

    def theta_history(self, cap_steps: int = 1 << 20) -> np.ndarray:
        """(steps, n_segments) sign-problem phase theta = atan2(Im N^diag,
        Re N^diag) after each step of the last ``step`` call, from the exact
        per-step N^diag the merge accumulates [End Matter, sign-problem
        suppression]."""
        h = self.step_history(cap_steps)
        return np.arctan2(h[:, :, 3].astype(np.float64), h[:, :, 2].astype(np.float64))

    def z_history(self, cap_steps: int = 1 << 20) -> np.ndarray:
        """(steps, n_segments, n_qubits) int64: N^diag <Z_q> after each step of
        the last ``step`` call (sum over the diagonal of Re N_xx (-1)^(x_q))."""
        buf = np.zeros((max(1, min(cap_steps, 1 << 22)), self.nseg, self.n), dtype=np.int64)
        cnt = C.c_int64()
        self._check(self.L.qmc_z_history(self.h, buf.ctypes.data, buf.shape[0], C.byref(cnt)), "qmc_z_history")
        return buf[:cnt.value]

    def overlap_all(self, psi: dict) -> np.ndarray:
        """complex (n_segments,): sum_ab conj(psi_a) N_ab psi_b of every vector."""
        idx = _arr(list(psi.keys()), np.uint64)
        vals = np.array([complex(v) for v in psi.values()])
        pr = _arr(vals.real, np.float64)
        pi = _arr(vals.imag, np.float64)
        orr = np.zeros(self.nseg, dtype=np.float64)
        oi = np.zeros(self.nseg, dtype=np.float64)
        self._check(self.L.qmc_overlap_all(self.h, _ptr(idx), _ptr(pr), _ptr(pi), len(idx), orr.ctypes.data,
                                           oi.ctypes.data), "qmc_overlap_all")
        return orr + 1j * oi

    def antihermiticity(self) -> list:
        """Exact ||N - N^dagger||_F^2 of every vector (Python ints)."""
        out = np.zeros(2 * self.nseg, dtype=np.uint64)
        self._check(self.L.qmc_antihermiticity(self.h, out.ctypes.data), "qmc_antihermiticity")
        return [int(out[2 * s]) + (int(out[2 * s + 1]) << 64) for s in range(self.nseg)]

    def antihermiticity_sum(self, vectors) -> int:
        """Exact ||S - S^dagger||_F^2 of the sum S of the listed vectors (a
        replica aggregate), a Python int."""
        v = _arr(list(vectors), np.int32)
        out = np.zeros(2, dtype=np.uint64)
        self._check(self.L.qmc_antihermiticity_sum(self.h, _ptr(v), len(v), out.ctypes.data),
                    "qmc_antihermiticity_sum")
        return int(out[0]) + (int(out[1]) << 64)

    def export(self, seg: int, which: int = 0):
        cnt = C.c_int64()
        rc = self.L.qmc_export(self.h, seg, which, None, None, None, 0, C.byref(cnt))
        if rc not in (OK, ERR_INVALID_ARG):
            self._check(rc, "qmc_export")
        n = cnt.value
        keys = np.zeros(n, dtype=np.uint64)
        re = np.zeros(n, dtype=np.int32)
        im = np.zeros(n, dtype=np.int32)
        self._check(self.L.qmc_export(self.h, seg, which, _ptr(keys), _ptr(re), _ptr(im), n, C.byref(cnt)),
                    "qmc_export")
        return keys, re, im

    def export_xy(self, seg: int, which: int = 0):
        """One vector's records as (x, y, re, im) in key order (any n)."""
        cnt = C.c_int64()
        rc = self.L.qmc_export_xy(self.h, seg, which, None, None, None, None, 0, C.byref(cnt))
        if rc not in (OK, ERR_INVALID_ARG):
            self._check(rc, "qmc_export_xy")
        n = cnt.value
        x = np.zeros(n, dtype=np.uint64)
        y = np.zeros(n, dtype=np.uint64)
        re = np.zeros(n, dtype=np.int32)
        im = np.zeros(n, dtype=np.int32)
        self._check(self.L.qmc_export_xy(self.h, seg, which, _ptr(x), _ptr(y), _ptr(re), _ptr(im), n, C.byref(cnt)),
                    "qmc_export_xy")
        return x, y, re, im

    def overlap(self, seg: int, psi: dict) -> complex:
        idx = _arr(list(psi.keys()), np.uint64)
        vals = np.array([complex(v) for v in psi.values()])
        pr = _arr(vals.real, np.float64)
        pi = _arr(vals.imag, np.float64)
        orr, oi = C.c_double(), C.c_double()
        self._check(self.L.qmc_overlap(self.h, seg, _ptr(idx), _ptr(pr), _ptr(pi), len(idx), C.byref(orr),
                                       C.byref(oi)), "qmc_overlap")
        return complex(orr.value, oi.value)

    def checkpoint(self, path: str):
        self._check(self.L.qmc_checkpoint(self.h, path.encode()), "qmc_checkpoint")

    def restore(self, path: str):
        self._check(self.L.qmc_restore(self.h, path.encode()), "qmc_restore")


def column_eval(prob, x: int, y: int, t: float, dt_eff: float, cap: int = 4096):
    """Host evaluation of the compiled column (qmc_column_eval): destinations in
    canonical order as (mask, re, im) in 2^-52 units, and the spawn weight P."""
    L = lib()
    ham = (HamTerm * max(1, len(prob.ham)))(*[HamTerm(h, xm, zm, r, w) for h, xm, zm, r, w in prob.ham])
    coefs, linds = [], []
    for ops, r, w in prob.lind:
        linds.append(Lindblad(len(coefs), len(ops), r, w))
        for coef, xm, zm in ops:
            coefs.append(PauliCoef(coef.real, coef.imag, xm, zm))
    lind = (Lindblad * max(1, len(linds)))(*linds)
    cf = (PauliCoef * max(1, len(coefs)))(*coefs)
    rates = (Rate * max(1, len(prob.rates)))(*[Rate(k, 0, a, b, c) for k, a, b, c in prob.rates])
    wins = (Window * max(1, len(prob.windows)))(*[Window(a, b) for a, b in prob.windows])
    mask = np.zeros(cap, dtype=np.uint64)
    mask_hi = np.zeros(cap, dtype=np.uint64)
    vre = np.zeros(cap, dtype=np.int64)
    vim = np.zeros(cap, dtype=np.int64)
    p = C.c_int64()
    vp = C.c_void_p
    L.qmc_column_eval.argtypes = [C.c_int32, vp, C.c_int32, vp, C.c_int32, vp, C.c_int32, vp, C.c_int32, vp,
                                  C.c_int32, C.c_double, C.c_double, C.c_uint64, C.c_uint64, C.c_int32, vp, vp, vp,
                                  vp, vp]
    L.qmc_column_eval.restype = C.c_int
    ne = L.qmc_column_eval(prob.n, ham, len(prob.ham), lind, len(linds), cf, len(coefs), rates, len(prob.rates),
                           wins, len(prob.windows), t, dt_eff, x, y, cap, mask.ctypes.data, mask_hi.ctypes.data,
                           vre.ctypes.data, vim.ctypes.data, C.byref(p))
    if ne < 0:
        raise QmcError(ne, "qmc_column_eval failed")
    if prob.n > 32:   # masks (dx << n) | dy of 2n > 64 bits as Python ints
        masks = np.array([(int(b) << 64) | int(a) for a, b in zip(mask[:ne], mask_hi[:ne])], dtype=object)
        return masks, vre[:ne], vim[:ne], p.value
    return mask[:ne], vre[:ne], vim[:ne], p.value
