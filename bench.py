"""Benchmark: walker-steps/s of the real-time population-dynamics QMC step.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gb300|reference]
                    [--workload spread32|spread32s|spread40|spread40s|dd12|dd12i|ghz4|ghzN|ghzNi|batch256]

One "step" is one dt step of every population vector through the whole hot
path: spawning (Hamiltonian and Lindblad terms, diagonal included), radix sort
of the spawns, annihilation + initiator rule + compaction, per-vector
observables.  value = sum over the timed steps of N_tot (walkers of N(t + dt),
all vectors, all ranks) / max-over-ranks device time.

Default workload ``spread32``: the 32-qubit GHZ Liouvillian (CNOT 4 -> 5
window, amplitude damping and dephasing on every qubit), 64 vectors holding
1e8 distinct random states of one walker each, dt = 0.01 (AB2), t from 5.0:
the working set (1.6 GB per population slot) is far larger than L2.  The other
workloads (dd12: staggered-XX dynamical decoupling on a 12-qubit ring, whose
populations fit in L2; ghzN: GHZ preparation from |0><0|) run the same path.

Multi-GPU: vectors are independent, so each rank runs its own 64 vectors
(seed offset by rank) with no collective on the data path ("weak" scaling).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2502_18929_gb300 import planner  # noqa: E402
from paper_2502_18929_gb300 import problems as P  # noqa: E402

METRIC = "walker-steps/s (spawn+annihilate)"
UNIT = "walker-steps/s"
L2_BYTES = 129 * 1024 * 1024


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return float(d.get("hbm_gbs", 6800.0)), "measured"
    return 6800.0, "fallback"


# ---------------------------------------------------------------------------
# workloads
# ---------------------------------------------------------------------------
def workload(name: str):
    if name in ("dd12", "dd12i"):
        prob = P.dd_ring(12, seed=0, t_end=20.0)
        xi = 1e-3 if name == "dd12i" else 0.0
        return dict(name=name, desc="staggered-XX DD, 12-qubit ring, ZZ crosstalk, X basis" +
                    (", initiator xi = 1e-3" if xi else ""),
                    prob=prob, nseg=64, n_diag=10**6, dt=0.005, t_end=20.0, rho0=P.rho_basis(0), xi=xi)
    if name == "ghz4":
        prob = P.ghz_circuit(4)
        return dict(name="ghz4", desc="GHZ-4 preparation", prob=prob, nseg=16, n_diag=10**4, dt=0.01,
                    t_end=4.0, rho0=P.rho_basis(0))
    if name.startswith("ghz") and name[3:].isdigit():
        n = int(name[3:])
        prob = P.ghz_circuit(n)
        total = {16: 10**7, 24: 5 * 10**7, 32: 10**8, 40: 10**8}.get(n, 10**7)
        # without the initiator the GHZ-24 walker number and its spawns per step grow several-fold
        return dict(name=name, desc=f"GHZ-{n} preparation", prob=prob, nseg=16, n_diag=total // 16, dt=0.01,
                    t_end=float(n), rho0=P.rho_basis(0), hint_factor=8 if n == 24 else 2)
    if name == "spread32":
        prob = P.ghz_circuit(32)
        return dict(name="spread32", desc="GHZ-32 Liouvillian (CNOT 4->5 window + local noise), "
                    "1e8 distinct random states x 1 walker over 64 vectors",
                    prob=prob, nseg=64, n_diag=10**8 // 64, dt=0.01, t_end=6.0, t_start=5.0,
                    spread=10**8 // 64, default_steps=10)
    if name == "spread40":
        prob = P.ghz_circuit(40)
        return dict(name="spread40", desc="GHZ-40 Liouvillian (CNOT 4->5 window + local noise), 128-bit keys, "
                    "1e8 distinct random states x 1 walker over 64 vectors",
                    prob=prob, nseg=64, n_diag=10**8 // 64, dt=0.01, t_end=6.0, t_start=5.0,
                    spread=10**8 // 64, default_steps=10)
    if name == "spread40s":
        prob = P.ghz_circuit(40)
        return dict(name="spread40s", desc="GHZ-40 Liouvillian (CNOT 4->5 window + local noise), 128-bit keys, "
                    "1.6e7 distinct random states x 1 walker over 64 vectors",
                    prob=prob, nseg=64, n_diag=250000, dt=0.01, t_end=6.0, t_start=5.0,
                    spread=250000, default_steps=10)
    if name == "spread32s":
        prob = P.ghz_circuit(32)
        return dict(name="spread32s", desc="GHZ-32 Liouvillian (CNOT 4->5 window + local noise), "
                    "1.6e7 distinct random states x 1 walker over 64 vectors",
                    prob=prob, nseg=64, n_diag=250000, dt=0.01, t_end=6.0, t_start=5.0,
                    spread=250000, default_steps=10)
    if name.startswith("ghz") and name.endswith("i") and name[3:-1].isdigit():
        n = int(name[3:-1])
        prob = P.ghz_circuit(n)
        total = {16: 10**7, 24: 5 * 10**7, 32: 10**8, 40: 10**8}.get(n, 10**7)
        return dict(name=name, desc=f"GHZ-{n} preparation, initiator xi = 1e-3", prob=prob, nseg=16,
                    n_diag=total // 16, dt=0.01, t_end=float(n), rho0=P.rho_basis(0), xi=1e-3)
    raise SystemExit(f"unknown workload {name}")


def capacity_hint(wl, nsteps: int) -> int:
    """Population slot capacity for a run of nsteps steps from the spread
    state: the records grow by about 1.3 % of the initial count per step in
    the CNOT window (new keys reached by spawns), so size for 2 % per step
    plus a quarter, and no buffer has to grow (and a step be redone) inside
    the timed region.  Workloads that start from a single state get two
    records per initial walker (a vector holds at most one record per walker,
    and without the initiator the walker number grows; `hint_factor` where it
    grows further), which also sizes the spawn buffer (a quarter of the
    hint)."""
    if "spread" not in wl:
        return int(wl["n_diag"] * wl["nseg"] * wl.get("hint_factor", 2))
    base = wl["spread"] * wl["nseg"]
    return int(base * (1.0 + 0.02 * nsteps) * 1.25)


def plan_steps(wl, warmup: int, steps: int):
    """(plan, total steps of the plan, timed steps K) for a run of `warmup`
    untimed and `steps` timed steps (0: the workload's default); raises
    SystemExit when the workload is shorter than warmup + steps."""
    pl = step_list(wl)
    total = planner.total_steps(pl)
    K = steps if steps > 0 else wl.get("default_steps", total - warmup)
    if warmup + K > total:
        raise SystemExit(f"workload {wl['name']} has {total} steps; warmup + steps = {warmup + K}")
    return pl, total, K


def host_inputs(wl, rank):
    """Synthetic inputs in pinned host memory (generated before any timing)."""
    import torch
    if "spread" not in wl:
        return None
    if wl["prob"].n > 32:
        pops = [P.spread_population_xy(wl["prob"].n, wl["spread"], 10 * s + rank) for s in range(wl["nseg"])]
        counts = np.array([len(p[0]) for p in pops], dtype=np.int64)
        cat = [torch.from_numpy(np.concatenate([p[k] for p in pops]).view(np.int64 if k < 2 else np.int32))
               .pin_memory() for k in range(4)]
        return ("xy", counts, *cat)
    pops = [P.spread_population(wl["prob"].n, wl["spread"], 10 * s + rank) for s in range(wl["nseg"])]
    counts = np.array([len(p[0]) for p in pops], dtype=np.int64)
    keys = torch.from_numpy(np.concatenate([p[0] for p in pops]).view(np.int64)).pin_memory()
    re = torch.from_numpy(np.concatenate([p[1] for p in pops])).pin_memory()
    im = torch.from_numpy(np.concatenate([p[2] for p in pops])).pin_memory()
    return counts, keys, re, im


def load_inputs(sim, wl, inputs):
    """Upload the inputs; returns the bytes copied host -> device."""
    if inputs is None:
        sim.init_populations(wl["rho0"])
        return len(wl["rho0"]) * 32
    if isinstance(inputs[0], str):   # ("xy", ...): more than 32 qubits, states as bit strings
        _, counts, x, y, re, im = inputs
        sim.set_populations_xy(counts, x.numpy().view(np.uint64), y.numpy().view(np.uint64), re.numpy(),
                               im.numpy())
        sim.set_clock(0, wl["t_start"])
        return int(x.numel() * 16 + re.numel() * 8 + counts.nbytes)
    counts, keys, re, im = inputs
    sim.set_populations_packed(counts, keys.numpy().view(np.uint64), re.numpy(), im.numpy())
    sim.set_clock(0, wl["t_start"])
    return int(keys.numel() * 8 + re.numel() * 4 + im.numel() * 4 + counts.nbytes)


def reduce_over_ranks(dist, values, device):
    """Whole-job figures of replicas: values = (ms, walker-steps, e2e seconds,
    e2e walker-steps) of this rank; returns the max of the times and the sum of
    the counts over all ranks (no data moves between ranks otherwise)."""
    import torch
    tt = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device)
    mx = tt.clone()
    dist.all_reduce(mx, op=dist.ReduceOp.MAX)
    sm_ = tt.clone()
    dist.all_reduce(sm_, op=dist.ReduceOp.SUM)
    return mx[0].item(), sm_[1].item(), mx[2].item(), sm_[3].item()


def set_proposal(sim, prob, kind: str):
    """Choice rule of the spawn step: the paper's exact rule, the static-weight
    proposal, the learned proposal with an untrained network (32 hidden units,
    static share 0.1), or the same on the tensor cores (64 hidden units, bf16,
    GELU)."""
    from paper_2502_18929_gb300 import qmc
    if kind == "static":
        sim.set_proposal(qmc.PROPOSAL_STATIC)
    elif kind == "learned":
        sim.set_mlp(P.random_network(prob, hidden=32, seed=0, eps=0.1))
        sim.set_proposal(qmc.PROPOSAL_LEARNED)
    elif kind == "learned_tc":
        sim.set_mlp(P.random_network(prob, hidden=64, seed=0, eps=0.1))
        sim.set_proposal(qmc.PROPOSAL_LEARNED_TC)


def piece_dt(pl, step: int) -> float:
    """Step size of the plan piece holding step `step`."""
    idx = 0
    for t0, d, n in pl:
        if step < idx + n:
            return d
        idx += n
    return pl[-1][1]


def run_e2e(wl, pl, inputs, nsteps, seed, init_min, stream, dist, tuning=None, proposal="exact"):
    import torch
    from paper_2502_18929_gb300 import qmc
    prob = wl["prob"]
    sim = qmc.QMC(prob.n, wl["nseg"], seed, wl["n_diag"], integrator=qmc.AB2, stream=stream.cuda_stream,
                  initiator_min=init_min, capacity_hint=capacity_hint(wl, nsteps))
    sim.load_schedule(prob)
    set_proposal(sim, prob, proposal)
    if tuning is not None:
        sim.set_tuning(**tuning)
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    t0 = time.perf_counter()
    h2d = load_inputs(sim, wl, inputs)
    d2h = 0
    walkers = 0
    idx = 0
    for tp0, d, n in pl:
        lo, hi = idx, idx + n
        idx = hi
        b = min(hi, nsteps)
        if lo >= b:
            break
        step, _, tpp, dl, pv = sim.clock()
        sim.set_clock(step, tp0, tpp, dl, pv)
        sim.step(d, b - lo)
        hist = sim.step_history()
        d2h += hist.nbytes
        walkers += int(hist[:, :, 1].sum())
        h2d += 0
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    sim.close()
    return {"seconds": t1 - t0, "walker_steps": walkers, "h2d_bytes": h2d, "d2h_bytes": d2h}


def step_list(wl):
    pl = planner.plan(wl["prob"], wl["t_end"], wl["dt"], t_start=wl.get("t_start", 0.0))
    return pl


def run_range(sim, pl, begin: int, count: int):
    """Steps [begin, begin + count) of plan pl (pieces keep their own dt)."""
    idx = 0
    done = 0
    for t0, d, n in pl:
        lo, hi = idx, idx + n
        idx = hi
        a, b = max(lo, begin), min(hi, begin + count)
        if a >= b:
            continue
        if a == lo:
            step, _, tp, dl, pv = sim.clock()
            sim.set_clock(step, t0, tp, dl, pv)
        sim.step(d, b - a)
        done += b - a
    return done


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.proc = None
        self.gpu = gpu_index
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(gpu_index), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except Exception:
            self.proc.kill()
            out = ""
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------
def source_sha() -> str:
    import hashlib
    src = b"".join(open(os.path.join(ROOT, "paper_2502_18929_gb300", "csrc", f), "rb").read()
                   for f in ("kernels.cu", "column_eval.h", "kernels.h", "qmc_types.h"))
    return hashlib.sha256(src).hexdigest()[:16]


def measured_traffic(kernel: str, units_launch: float):
    """DRAM bytes (read + write) of one launch of `kernel`, scaled by the units
    processed (parents plus spawn candidates for the draw kernel; merged items
    plus outputs for the merge) from the ncu counters kept as data in
    profiles/<kernel>_spread32s.json.  None when no capture exists or the
    kernel sources changed since it was taken."""
    path = os.path.join(ROOT, "profiles", f"{kernel}_spread32s.json")
    if not os.path.exists(path):
        return None
    with open(path) as f:
        d = json.load(f)
    if d.get("kernel_sources_sha256_16") != source_sha() or not d.get("units_of_launch"):
        return None
    m = d["metrics"]
    scale = {"byte": 1.0, "Kbyte": 1e3, "Mbyte": 1e6, "Gbyte": 1e9}
    total = 0.0
    for key in ("dram__bytes_read.sum", "dram__bytes_write.sum"):
        if key not in m:
            return None
        total += float(m[key]["value"]) * scale.get(m[key]["unit"], 1.0)
    return total * units_launch / float(d["units_of_launch"])


def kernel_bytes(name: str, c: dict) -> float:
    """Algorithmic bytes of a kernel over the counted steps (16-byte records)."""
    r = 16.0
    lsd = c.get("sort_lsd_steps", 0) / max(1, c["steps"])   # share of steps on the LSD sort
    if name == "k_spawn_draw":     # parents read, candidates written
        return r * (c["k_cur"] + c["k_prev"] + c["candidates"])
    if name == "k_spawn_choose":   # candidates and their parents' keys read, spawn records written
        return (r + 8.0) * c["candidates"] + r * c["spawns"]
    if name == "k_merge":
        return r * (c["k_cur"] + c["spawns"] + c["k_next"])
    if name == "k_bucket_hist":
        return r * c["spawns"] * (1.0 - lsd)
    if name in ("k_bucket_scatter", "k_bucket_sort"):
        return 2.0 * r * c["spawns"] * (1.0 - lsd)
    if name == "k_sort_scatter":
        return 2.0 * r * c["spawns"] * c.get("passes", 1) * lsd
    if name == "k_sort_hist":
        return r * c["spawns"] * lsd
    return 0.0


def run_gpu(args, rank: int, world: int):
    import torch
    from paper_2502_18929_gb300 import qmc

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    torch.cuda.init()
    dist = None
    if world > 1:
        import torch.distributed as tdist
        tdist.init_process_group("nccl", device_id=torch.device("cuda", local))
        dist = tdist
    wl = workload(args.workload)
    prob = wl["prob"]
    stream = torch.cuda.current_stream()
    seed = 1000 + rank
    init_min = int(math.ceil(wl.get("xi", 0.0) * wl["n_diag"]))
    W = args.warmup
    pl, total, K = plan_steps(wl, W, args.steps)
    sim = qmc.QMC(prob.n, wl["nseg"], seed, wl["n_diag"], integrator=qmc.AB2, stream=stream.cuda_stream,
                  initiator_min=init_min, capacity_hint=capacity_hint(wl, W + K))
    sim.load_schedule(prob)
    set_proposal(sim, prob, args.proposal)

    inputs = host_inputs(wl, rank)
    load_inputs(sim, wl, inputs)
    run_range(sim, pl, 0, W)
    torch.cuda.synchronize()
    tuning = None
    if args.autotune:
        # launch shapes timed from the warmed-up state, which the tuner restores
        tuning = sim.autotune(piece_dt(pl, W), 3)
    sim.counters(reset=True)
    nkeys_start = int(sim.observables()[:, 0].sum())

    ck_path = None
    wide = prob.n > 32
    if not args.no_profile and not wide:
        import tempfile
        ck_path = os.path.join(tempfile.gettempdir(), f"qmc_bench_ck_{os.getpid()}_{rank}.bin")
        sim.checkpoint(ck_path)

    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    sampler = ClockSampler(local)
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    t_wall0 = time.perf_counter()
    ev0.record(stream)
    run_range(sim, pl, W, K)
    ev1.record(stream)
    torch.cuda.synchronize()
    t_wall1 = time.perf_counter()
    clocks = sampler.stop()
    if dist is not None:
        dist.barrier()
    ms = ev0.elapsed_time(ev1)
    c = sim.counters(reset=True)
    walkers = c["walker_steps"]
    if c["redo_launches"]:
        raise SystemExit(f"{c['redo_launches']} step launches were redone inside the timed region "
                         "(a buffer grew): raise the capacity hint")
    launches_per_step = sim.step_launches()   # the step graph as timed (same buffers)

    # per-kernel times over the same timed steps (replayed from the checkpoint)
    roof = None
    kernel_ms = {}
    if ck_path is not None:
        sim.restore(ck_path)
        sim.counters(reset=True)
        idx = 0
        for t0, d, n in pl:
            lo, hi = idx, idx + n
            idx = hi
            a, b = max(lo, W), min(hi, W + K)
            if a >= b:
                continue
            if a == lo:
                step, _, tp, dl, pv = sim.clock()
                sim.set_clock(step, t0, tp, dl, pv)
            for name, v in sim.step_profile(d, b - a).items():
                kernel_ms[name] = kernel_ms.get(name, 0.0) + v
        cp = sim.counters(reset=True)
        cp["passes"] = (2 * prob.n + 7) // 8 + (math.ceil(math.log2(wl["nseg"])) + 7) // 8
        try:
            os.remove(ck_path)
        except OSError:
            pass
        peak, peak_kind = load_peaks()
        top = max(kernel_ms, key=kernel_ms.get)
        launches = cp["steps"] * (cp["passes"] if top == "k_sort_scatter" else 1)
        avg_ms = kernel_ms[top] / max(1, launches)
        bytes_per_launch = kernel_bytes(top, cp) / max(1, launches)
        achieved = bytes_per_launch / (avg_ms * 1e-3) / 1e9 if avg_ms > 0 else 0.0
        unit_counts = {"k_spawn_draw": (cp["k_cur"] + cp["k_prev"] + cp["candidates"]) / max(1, cp["steps"]),
                       "k_merge": (cp["k_cur"] + cp["spawns"] + cp["k_next"]) / max(1, cp["steps"])}
        units = unit_counts.get(top, 0) * cp["steps"] / max(1, launches)
        traffic = measured_traffic(top, units) if units else None
        roof = {"bound": "hbm", "kernel": top, "achieved": round(achieved, 1), "peak": peak,
                "peak_kind": peak_kind, "unit": "GB/s", "frac": round(achieved / peak, 4),
                "traffic": None if traffic is None else round(traffic),
                "traffic_source": (None if traffic is None else
                                   f"ncu DRAM read + write of {top} on spread32s (profiles/{top}_spread32s.json), "
                                   "scaled to this launch by the units processed"),
                "avg_launch_ms": round(avg_ms, 5),
                "algorithmic_bytes_per_launch": round(bytes_per_launch),
                "units_per_launch": {k: round(v) for k, v in unit_counts.items()},
                "kernel_share": {k: round(v / sum(kernel_ms.values()), 4) for k, v in kernel_ms.items()}}

    if wide:
        # the whole step against the bytes it cannot avoid, 24-byte records
        # read by the spawn pass (N(t), N(t - dt)) and the merge (N(t)), spawns
        # written and read once, N(t + dt) written; the kernel groups' shares
        # from three further steps replayed under events
        peak, peak_kind = load_peaks()
        if not args.no_profile and W + K + 3 <= total:
            idx = 0
            for t0, d, n in pl:
                lo, hi = idx, idx + n
                idx = hi
                a, b = max(lo, W + K), min(hi, W + K + 3)
                if a >= b:
                    continue
                if a == lo:
                    step, _, tp, dl, pv = sim.clock()
                    sim.set_clock(step, t0, tp, dl, pv)
                for name, v in sim.step_profile(d, b - a).items():
                    kernel_ms[name] = kernel_ms.get(name, 0.0) + v
        steps = max(1, c["steps"])
        bytes_step = 24.0 * (2 * c["k_cur"] + c["k_prev"] + 2 * c["spawns"] + c["k_next"]) / steps
        achieved = bytes_step / (ms / K * 1e-3) / 1e9
        roof = {"bound": "hbm", "kernel": "whole step (128-bit keys)", "achieved": round(achieved, 1),
                "peak": peak, "peak_kind": peak_kind, "unit": "GB/s", "frac": round(achieved / peak, 4),
                "traffic": None, "algorithmic_bytes_per_step": round(bytes_step)}
        if kernel_ms:
            roof["kernel_share"] = {k: round(v / sum(kernel_ms.values()), 4) for k, v in kernel_ms.items()}

    # end to end through the public API: a fresh context, inputs uploaded from
    # pinned host memory, every step, and a D2H read of each call's per-step
    # observables (the step's result), timed on the host clock
    sim.close()
    e2e = run_e2e(wl, pl, inputs, W + K, seed, init_min, stream, dist, tuning, args.proposal)
    if dist is not None:
        ms_all, walkers_all, e2e_s, e2e_w = reduce_over_ranks(
            dist, (ms, float(walkers), e2e["seconds"], float(e2e["walker_steps"])), "cuda")
    else:
        ms_all, walkers_all, e2e_s, e2e_w = ms, float(walkers), e2e["seconds"], float(e2e["walker_steps"])

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        cpu = cpu_baseline(wl, budget_s=args.cpu_budget, all_cores=not args.cpu_single)

    if rank != 0:
        return
    value = walkers_all / (ms_all * 1e-3)
    ws = 3 * c["k_next"] / max(1, c["steps"]) * (24 if wide else 16) * (world if world > 1 else 1)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K, "warmup": W,
        "ms_per_step": ms_all / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "int64", "data": "synthetic",
        "config": {"workload": wl["name"], "description": wl["desc"], "n_qubits": prob.n,
                   "vectors_per_gpu": wl["nseg"], "n_diag": wl["n_diag"], "dt": wl["dt"],
                   "integrator": "AB2", "xi": wl.get("xi", 0.0), "timed_steps_of_job": f"{W}..{W + K} of {total}",
                   "records_per_step_avg": c["k_next"] / max(1, c["steps"]),
                   "spawns_per_step_avg": c["spawns"] / max(1, c["steps"]),
                   "key_steps_per_s": c["k_next"] * world / (ms_all * 1e-3),
                   "l2": ("inputs larger than L2" if ws > L2_BYTES else
                          "working set below L2 (no flush between steps)"),
                   "parallelism": f"replicas x{world}",
                   "launch_shapes": tuning if tuning is not None else "default",
                   "proposal": args.proposal, "redo_launches_timed": c["redo_launches"]},
        "e2e": {"value": e2e_w / e2e_s, "unit": UNIT, "h2d_bytes_per_step": e2e["h2d_bytes"] / (W + K),
                "d2h_bytes_per_step": e2e["d2h_bytes"] / (W + K), "steps": W + K,
                "includes": "input upload from pinned host memory, all warm-up and timed steps, "
                            "D2H of per-step observables after every call"},
        "gpu_launches": int(c["steps"] * launches_per_step),
        "clocks": clocks,
    }
    if roof is not None:
        line["roofline"] = roof
    if cpu is not None:
        line["cpu_baseline"] = cpu
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# Batched step: many independent problem instances in one context
# ---------------------------------------------------------------------------
def batch_instances(k: int = 256, seed: int = 0):
    """GHZ circuits, n ~ U{4..16}, amplitude damping and dephasing at
    gamma0 cos(omega t) with gamma0 ~ U[0.01, 0.05], omega ~ U[0.5, 2],
    N^diag log-uniform in [1e4, 1e6], one vector each."""
    rng = np.random.default_rng(seed)
    probs, ndiag, seeds = [], [], []
    for i in range(k):
        n = int(rng.integers(4, 17))
        g0 = float(rng.uniform(0.01, 0.05))
        om = float(rng.uniform(0.5, 2.0))
        probs.append(P.ghz_circuit(n, gamma1=g0, gamma_phi=g0, rate_kind=P.RATE_COS, omega1=om, omega_phi=om))
        ndiag.append(int(10 ** rng.uniform(4.0, 6.0)))
        seeds.append(7 * i + 1)
    return probs, ndiag, seeds


def run_batch(args, rank: int, world: int):
    """256 instances stepped by one context (qmc_batch_create), against the
    same instances stepped one context each, one after the other.  Both start
    from |0><0| and pre-roll 100 steps (t = 1, the end of the Hadamard pulse)
    untimed; then W warm-up and K timed steps of dt = 0.01."""
    import torch
    from paper_2502_18929_gb300 import qmc
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    torch.cuda.init()
    stream = torch.cuda.current_stream()
    probs, ndiag, seeds = batch_instances(256, rank)
    k = len(probs)
    dt, pre, W = 0.01, 100, max(3, args.warmup)
    K = args.steps if args.steps > 0 else 20
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def timed(sim, nsteps):
        torch.cuda.synchronize()
        h0 = time.perf_counter()
        ev0.record(stream)
        sim.step(dt, nsteps)
        ev1.record(stream)
        torch.cuda.synchronize()
        return ev0.elapsed_time(ev1), time.perf_counter() - h0

    batch = qmc.QMC.batch(probs, [1] * k, seeds, ndiag, stream=stream.cuda_stream)
    batch.init_populations(P.rho_basis(0))
    batch.step(dt, pre + W)
    batch.counters(reset=True)
    sampler = ClockSampler(local)
    ms, host_s = timed(batch, K)
    clocks = sampler.stop()
    c = batch.counters(reset=True)
    launches = batch.step_launches()
    prof = batch.step_profile(dt, 3)   # three further steps replayed under events
    tot = sum(prof.values()) or 1.0
    shares = {name: round(v / tot, 4) for name, v in sorted(prof.items(), key=lambda kv: -kv[1]) if v > 0}
    batch.close()

    alone_ms, alone_host, alone_walkers = 0.0, 0.0, 0
    for i in range(k):
        sim = qmc.QMC(probs[i].n, 1, seeds[i], ndiag[i], stream=stream.cuda_stream)
        sim.load_schedule(probs[i])
        sim.init_populations(P.rho_basis(0))
        sim.step(dt, pre + W)
        sim.counters(reset=True)
        m, h = timed(sim, K)
        alone_ms += m
        alone_host += h
        alone_walkers += sim.counters()["walker_steps"]
        sim.close()
    if alone_walkers != c["walker_steps"]:
        raise SystemExit("batched and per-instance runs disagree on the walker count")

    # the strongest plain form: one context per instance, 16 host threads each
    # stepping 16 contexts on its own stream, all at once (host wall time)
    from concurrent.futures import ThreadPoolExecutor
    nthreads = 16
    streams = [torch.cuda.Stream() for _ in range(nthreads)]
    sims = []
    for i in range(k):
        sm = qmc.QMC(probs[i].n, 1, seeds[i], ndiag[i], stream=streams[i % nthreads].cuda_stream)
        sm.load_schedule(probs[i])
        sm.init_populations(P.rho_basis(0))
        sm.step(dt, pre + W)
        sm.counters(reset=True)
        sims.append(sm)
    torch.cuda.synchronize()

    def worker(tix):
        for i in range(tix, k, nthreads):
            sims[i].step(dt, K)

    h0 = time.perf_counter()
    with ThreadPoolExecutor(nthreads) as ex:
        list(ex.map(worker, range(nthreads)))
    torch.cuda.synchronize()
    conc_s = time.perf_counter() - h0
    conc_walkers = sum(sm.counters()["walker_steps"] for sm in sims)
    for sm in sims:
        sm.close()
    if conc_walkers != c["walker_steps"]:
        raise SystemExit("batched and concurrent per-instance runs disagree on the walker count")
    value = c["walker_steps"] / (ms * 1e-3)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K, "warmup": W,
        "ms_per_step": ms / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "int64", "data": "synthetic",
        "config": {"workload": "batch256",
                   "description": "256 GHZ instances (n 4..16, cos-modulated damping and dephasing, N^diag "
                                  "1e4..1e6, one vector each) stepped by one context",
                   "n_qubits": "4..16", "instances": k, "dt": dt, "integrator": "AB2",
                   "timed_steps_of_job": f"{pre + W}..{pre + W + K}",
                   "records_per_step_avg": c["k_next"] / max(1, c["steps"]),
                   "spawns_per_step_avg": c["spawns"] / max(1, c["steps"]),
                   "parallelism": f"replicas x{world}"},
        "e2e": {"value": c["walker_steps"] / host_s, "unit": UNIT, "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0,
                "includes": "host time of the qmc_step call (column programs of every instance and step, "
                            "upload, graph launches)"},
        "unbatched": {"value": alone_walkers / (alone_ms * 1e-3), "unit": UNIT,
                      "ms_per_step": alone_ms / K, "host_s": alone_host,
                      "note": "the same 256 instances, one context each, stepped one after the other"},
        "unbatched_concurrent": {"value": conc_walkers / conc_s, "unit": UNIT, "host_s": conc_s,
                                 "note": f"one context per instance, {nthreads} host threads and streams, "
                                         "stepped concurrently (host wall time)"},
        "kernel_share": shares,
        "batched_speedup": (alone_ms / ms) if ms > 0 else None,
        "batched_speedup_vs_concurrent": (conc_s / host_s) if host_s > 0 else None,
        "gpu_launches": int(K * launches),
        "clocks": clocks,
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# CPU oracle (cpu_baseline leg and --impl reference)
# ---------------------------------------------------------------------------
CPU_SAMPLE_STATES = 50000   # states of one spread-workload vector in a CPU sample


def cpu_info() -> dict:
    """Host CPU model and the cores this process may use."""
    model = None
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                k, _, v = line.partition(":")
                if k.strip() in ("model name", "Model name") and v.strip():
                    model = v.strip()
                    break
    except OSError:
        pass
    if model is None:
        try:
            out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
            for line in out.splitlines():
                k, _, v = line.partition(":")
                if k.strip() == "Model name" and v.strip():
                    model = v.strip()
                    break
        except Exception:
            pass
    try:
        nproc = len(os.sched_getaffinity(0))
    except AttributeError:
        nproc = os.cpu_count() or 1
    import platform
    return {"cpu_model": model or platform.processor() or "unknown", "nproc": nproc,
            "machine": platform.machine()}


def oracle_vector(name: str, vec: int, budget_s: float):
    """One vector of workload `name` stepped by the oracle, single-threaded,
    until `budget_s` seconds have passed (whole steps): returns (walker-steps,
    seconds, steps).  Spread workloads take CPU_SAMPLE_STATES random states of
    the same distribution at the same time; the others start from their
    initial state.  Module-level so a spawned worker process can run it."""
    from oracle import oracle as O
    wl = workload(name)
    pl = step_list(wl)
    prob = wl["prob"]
    sim = O.OracleSim(prob, 1, 1000 + vec, integrator=O.AB2, n_diag=wl["n_diag"])
    if "spread" in wl:
        x, y, r, i = P.spread_population_xy(prob.n, min(wl["spread"], CPU_SAMPLE_STATES), 10 * vec)
        sim.set_population_xy(0, x, y, r, i)
        sim.set_clock(0, wl["t_start"])
    else:
        sim.init(wl["rho0"])
    t0 = time.perf_counter()
    walkers = 0
    steps = 0
    for tp0, d, n in pl:
        for j in range(n):
            if j == 0:
                stp, _, tpp, dl, pv = sim.clock()
                sim.set_clock(stp, tp0, tpp, dl, pv)
            rc = sim.step(d, 1)
            if rc != 0:
                raise RuntimeError(f"oracle step failed {rc}")
            walkers += int(sim.stats(0)[1])
            steps += 1
            if time.perf_counter() - t0 > budget_s:
                break
        if time.perf_counter() - t0 > budget_s:
            break
    return walkers, time.perf_counter() - t0, steps


def _oracle_worker(a):
    return oracle_vector(*a)


def cpu_baseline(wl, budget_s: float = 15.0, all_cores: bool = True):
    """The oracle as it stands on the host cores: one vector single-threaded,
    and (all_cores) one vector per core in spawned worker processes (vectors
    are independent, so this is the thread-per-vector form; the workers start
    with the spawn method and share nothing with this process's CUDA state).
    Each leg runs whole steps until its budget is used."""
    info = cpu_info()
    w1, s1, n1 = oracle_vector(wl["name"], 0, budget_s)
    states = f"{min(wl['spread'], CPU_SAMPLE_STATES)} random states" if "spread" in wl else "its initial state"
    sample = (f"1 vector of {wl['name']} from {states}, first {n1} steps (Euler, then AB2), "
              f"{s1:.1f} s")
    res = {"value": w1 / s1, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample,
           "cpu_model": info["cpu_model"], "nproc": info["nproc"], "machine": info["machine"]}
    if all_cores and info["nproc"] > 1:
        import multiprocessing as mp
        nw = info["nproc"]
        with mp.get_context("spawn").Pool(nw) as pool:
            out = pool.map(_oracle_worker, [(wl["name"], v, budget_s) for v in range(nw)])
        wa = sum(o[0] for o in out)
        sa = max(o[1] for o in out)
        res["all_cores"] = {"value": wa / sa, "unit": UNIT, "cores": nw, "kind": "oracle",
                            "sample": f"{nw} vectors, one per worker process, each from {states}, "
                                      f"{min(o[2] for o in out)}-{max(o[2] for o in out)} steps, "
                                      f"{sa:.1f} s wall"}
    return res


def run_reference(args, rank: int, world: int):
    """The oracle as the reference arm: rank 0 alone, all host cores (one
    vector per worker process), each worker running whole steps for a budget
    that keeps the run within a few minutes."""
    if rank != 0:
        return
    wl = workload(args.workload)
    W = args.warmup
    pl, total, K = plan_steps(wl, W, args.steps)
    budget = max(5.0, min(60.0, 4.0 * (K + W)))
    res = cpu_baseline(wl, budget_s=budget, all_cores=True)
    arm = res.get("all_cores", res)
    cpu = dict(arm)
    cpu.update({"cpu_model": res["cpu_model"], "nproc": res["nproc"], "single_core": res["value"],
                "single_core_sample": res["sample"]})
    line = {"impl": "reference", "metric": METRIC, "value": arm["value"], "unit": UNIT, "n_gpus": world,
            "steps": K, "warmup": W, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "int64", "data": "synthetic",
            "config": {"workload": wl["name"], "description": wl["desc"]},
            "cpu_baseline": cpu,
            "e2e": {"value": arm["value"], "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=0, help="timed steps (0 = rest of the job)")
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default="spread32")
    ap.add_argument("--no-profile", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--proposal", default="exact", choices=["exact", "static", "learned", "learned_tc"],
                    help="spawn choice rule (learned: an untrained network)")
    ap.add_argument("--autotune", action="store_true",
                    help="time candidate launch shapes after the warm-up (state kept) and use the fastest")
    ap.add_argument("--cpu-budget", type=float, default=15.0)
    ap.add_argument("--cpu-single", action="store_true", help="cpu_baseline: skip the all-core oracle leg")
    args = ap.parse_args()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if args.impl == "reference":
        run_reference(args, rank, world)
    elif args.workload == "batch256":
        run_batch(args, rank, world)
    else:
        run_gpu(args, rank, world)


if __name__ == "__main__":
    main()
