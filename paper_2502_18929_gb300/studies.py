"""Measurement studies built on the library (GPU): the initiator bias and its
xi -> 0 extrapolation, and replica aggregation with the paper's scaling fits.

    python -m paper_2502_18929_gb300.studies initiator --out initiator.json
    python -m paper_2502_18929_gb300.studies replicas --out replicas.json
    python -m paper_2502_18929_gb300.studies proposal --workload ghz24 --out proposal.json

* Initiator study [End Matter, simulation methodology: spawns of parents
  below xi N^diag onto unoccupied states are discarded; the truncation error
  extrapolates to zero as xi -> 0]: GHZ preparation under local noise, final
  fidelity to the GHZ state and N^diag per vector for several xi, the
  weighted linear extrapolation of the fidelity to xi = 0, and the step
  throughput.
* Replica study [Markovian circuit dynamics: replica aggregation with
  N^diag_eff = r N^diag; dim(H_QMC) and its fit; End Matter on Hermiticity
  preservation]: staggered-XX DD from |+>^n (X basis) or |W>_n, r replicas
  per size, per-replica and aggregate fidelity and trace with bootstrap 95 %
  intervals, the occupied-state count of aggregates, the aggregate's
  anti-Hermiticity, and the fits of both models.
"""
from __future__ import annotations

import argparse
import json
import math
import time

import numpy as np

from . import analysis as A
from . import planner
from . import problems as P
from . import qmc


def run_vectors(prob, t_end: float, dt: float, nvec: int, n_diag: int, seed: int, rho0, xi: float = 0.0,
                target=None, capacity_hint: int = 0):
    """Step nvec vectors of one problem from rho0 to t_end (planned pieces)
    and return per-vector final results, the steps' device time and
    walker-steps."""
    import torch
    init_min = int(math.ceil(xi * n_diag))
    sim = qmc.QMC(prob.n, nvec, seed, n_diag, integrator=qmc.AB2, initiator_min=init_min,
                  capacity_hint=capacity_hint, stream=torch.cuda.current_stream().cuda_stream)
    sim.load_schedule(prob)
    sim.init_populations(rho0)
    pl = planner.plan(prob, t_end, dt)
    sim.counters(reset=True)
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record()
    planner.run(sim, pl)
    ev1.record()
    torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1)
    c = sim.counters()
    obs = sim.observables()
    out = {"records": obs[:, 0].tolist(), "n_tot": obs[:, 1].tolist(), "n_diag_re": obs[:, 2].tolist(),
           "n_diag_im": obs[:, 3].tolist(), "ms": ms, "walker_steps": c["walker_steps"], "steps": c["steps"],
           "antiherm": [str(v) for v in sim.antihermiticity()]}
    if target is not None:
        ov = sim.overlap_all(target)
        norm = sum(abs(complex(v)) ** 2 for v in target.values())
        out["overlap_re"] = (ov.real / norm).tolist()
        out["overlap_im"] = (ov.imag / norm).tolist()
    out["sim"] = sim
    return out


def extrapolate(xis, means, ses) -> dict:
    """Weighted least squares of F(xi) = F0 + a xi over xi > 0; F0 and its
    standard error."""
    x = np.asarray(xis, dtype=np.float64)
    y = np.asarray(means, dtype=np.float64)
    w = 1.0 / np.asarray(ses, dtype=np.float64) ** 2
    M = np.stack([np.ones_like(x), x], axis=1)
    cov = np.linalg.inv(M.T @ (w[:, None] * M))
    coef = cov @ (M.T @ (w * y))
    return {"F0": float(coef[0]), "se": float(math.sqrt(cov[0, 0])), "slope": float(coef[1])}


def initiator_study(sizes=(8, 16, 24, 32), xis=(1e-2, 3e-3, 1e-3, 3e-4, 0.0), nvec: int = 16,
                    n_diag: int = 10**5, seed: int = 11, dt: float = 0.01, zero_max_n: int = 16):
    """Final GHZ fidelity and N^diag per (n, xi), the xi -> 0 extrapolation
    per n, and walker-steps/s.  xi = 0 is run only up to zero_max_n qubits
    (without the initiator the larger circuits hit the sign problem: their
    walker number outgrows the buffers)."""
    rows = []
    for n in sizes:
        prob = P.ghz_circuit(n)
        target = P.ghz_target(n)
        pts = []
        for xi in xis:
            if xi == 0.0 and n > zero_max_n:
                continue
            r = run_vectors(prob, float(n), dt, nvec, n_diag, seed, P.rho_basis(0), xi=xi, target=target)
            nd = np.asarray(r["n_diag_re"], dtype=np.float64)
            fid = np.abs(np.asarray(r["overlap_re"]) + 1j * np.asarray(r["overlap_im"])) / n_diag
            row = {"n": n, "xi": xi, "fidelity": float(fid.mean()), "fidelity_se": float(fid.std(ddof=1) / math.sqrt(nvec)),
                   "trace": float(nd.mean() / n_diag), "trace_se": float(nd.std(ddof=1) / math.sqrt(nvec) / n_diag),
                   "records_final": float(np.mean(r["records"])), "ms": r["ms"], "steps": r["steps"],
                   "walker_steps_per_s": r["walker_steps"] / (r["ms"] * 1e-3)}
            rows.append(row)
            pts.append(row)
            r["sim"].close()
        fit = [p for p in pts if p["xi"] > 0]
        if len(fit) >= 2:
            ex = extrapolate([p["xi"] for p in fit], [p["fidelity"] for p in fit], [p["fidelity_se"] for p in fit])
            for p in pts:
                p["extrapolated_F0"] = ex["F0"]
                p["extrapolated_se"] = ex["se"]
    return rows


def _union_records(sim, segs) -> int:
    keys = [sim.export(s)[0] for s in segs]
    return int(np.unique(np.concatenate(keys)).size) if keys else 0


def replica_study(sizes=(8, 10, 12, 14), state: str = "plus", replicas: int = 5, n_diag: int = 2 * 10**5,
                  seed: int = 5, t_end: float = 4.0, dt: float = 0.005, xi: float = 0.0):
    """Replica aggregation on the staggered-XX DD ring (|+>^n in the X basis
    or |W>_n): per size, r replicas of N^diag walkers; aggregates of 2 .. r
    replicas give N^diag_eff = 2 .. r times N^diag.  xi > 0 runs with the
    initiator (the W state in the computational basis has a sign problem at
    these walker numbers without it)."""
    rows = []
    for n in sizes:
        if state == "plus":
            prob = P.dd_ring(n, seed=0, t_end=t_end, x_basis=True)
            rho0, target = P.rho_basis(0), {0: 1.0}
        else:
            prob = P.dd_ring(n, seed=0, t_end=t_end, x_basis=False)
            rho0, target = P.rho_pure(P.w_state(n)), P.w_state(n)
        r = run_vectors(prob, t_end, dt, replicas, n_diag, seed, rho0, xi=xi, target=target)
        sim = r["sim"]
        ov = np.asarray(r["overlap_re"]) + 1j * np.asarray(r["overlap_im"])
        nd = np.asarray(r["n_diag_re"], dtype=np.float64)
        fid = np.abs(ov) / n_diag
        est, lo, hi = A.bootstrap_ci(fid)
        row = {"n": n, "state": state, "replicas": replicas, "n_diag": n_diag, "xi": xi,
               "fidelity_per_replica": fid.tolist(), "fidelity_mean": float(est), "fidelity_ci95": [float(lo), float(hi)],
               "trace_per_replica": (nd / n_diag).tolist(),
               "ms": r["ms"], "walker_steps_per_s": r["walker_steps"] / (r["ms"] * 1e-3), "aggregates": []}
        for k in range(2, replicas + 1):
            segs = list(range(k))
            agg = A.aggregate(ov[:k], n_diag)
            tr = A.aggregate(nd[:k], n_diag)
            frob2 = sim.antihermiticity_sum(segs)
            row["aggregates"].append({"replicas": k, "n_diag_eff": agg["n_diag_eff"],
                                      "fidelity": float(abs(agg["estimate"])), "trace": float(tr["estimate"]),
                                      "dim_h_qmc": _union_records(sim, segs),
                                      "epsilon": A.antiherm_epsilon(frob2, agg["n_diag_eff"])})
        sim.close()
        rows.append(row)
    pts = [(row["n"], a["n_diag_eff"], a["dim_h_qmc"], a["epsilon"]) for row in rows for a in row["aggregates"]]
    fits = {}
    if len({p[0] for p in pts}) >= 2:
        n_, nd_, dim_, eps_ = (np.array(v, dtype=np.float64) for v in zip(*pts))
        fits["subspace"] = A.fit_subspace(n_, nd_, dim_)
        fits["antiherm"] = A.fit_antiherm(n_, nd_, eps_)
        fits["n_diag_opt_tau_0.02"] = {str(int(n)): A.n_diag_opt(float(n), 0.02, fits["antiherm"])
                                       for n in sorted({p[0] for p in pts})}
    return {"rows": rows, "fits": fits}


def _final_fidelity(sim, target, n_diag):
    ov = sim.overlap_all(target)
    norm = sum(abs(complex(v)) ** 2 for v in target.values())
    return np.abs(ov / norm) / n_diag


def proposal_study(name: str = "ghz24", nvec: int = 32, n_diag: int = 10**5, train_events: int = 10**7,
                   train_steps: int = 300, hidden: int = 64, eps: float = 0.1, t_end: float | None = None,
                   seed: int = 3):
    """The learned proposal against the static and the exact rule [A9; the
    library's extension].  Training: events logged from a run of the exact
    rule (heat-bath shares of every present destination, weighted by the
    parent's walkers) until train_events are collected, then full-batch Adam
    on the tensor cores.  Comparison: nvec vectors of n_diag walkers per rule
    from the same initial state; the final fidelity's spread over vectors s
    gives the walkers needed for a standard error of 10^-3, n_diag (s /
    10^-3)^2, and the time to reach it, time (s / 10^-3)^2 / nvec."""
    import torch
    from . import train as TR
    if name.startswith("dd"):
        n = int(name[2:].rstrip("i"))
        prob = P.dd_ring(n, seed=0, t_end=t_end or 4.0, x_basis=True)
        rho0, target, dt, xi = P.rho_basis(0), {0: 1.0}, 0.005, 1e-3
        t_end = t_end or 4.0
    else:
        n = int(name[3:].rstrip("i"))
        prob = P.ghz_circuit(n)
        rho0, target, dt, xi = P.rho_basis(0), P.ghz_target(n), 0.01, 1e-3 if name.endswith("i") else 0.0
        t_end = t_end or float(n)
    net = P.random_network(prob, hidden=hidden, seed=seed, eps=eps)
    pl = planner.plan(prob, t_end, dt)
    init_min = int(math.ceil(xi * n_diag))
    # events from the exact rule
    sim = qmc.QMC(prob.n, nvec, seed, n_diag, integrator=qmc.AB2, initiator_min=init_min)
    sim.load_schedule(prob)
    sim.set_mlp(net)
    sim.init_populations(rho0)
    t0 = time.time()
    feats, targets, weights, total = [], [], [], 0
    steps_total = planner.total_steps(pl)
    every = max(1, steps_total // 400)   # about 400 logging points over the run
    idx = 0
    for tp0, d, k in pl:
        done = 0
        step, _, tpp, dl, pv = sim.clock()
        sim.set_clock(step, tp0, tpp, dl, pv)
        while done < k:
            if total < train_events:
                f, tg, w, ne = sim.learn_events(d, min(1 << 20, train_events - total))
                feats.append(f[:, :ne])
                targets.append(tg[:, :ne])
                weights.append(w[:ne])
                total += ne
            m = min(every, k - done)
            sim.step(d, m)
            done += m
        idx += k
    sim.close()
    feat = torch.cat(feats, dim=1).contiguous()
    target_t = torch.cat(targets, dim=1).contiguous()
    weight = torch.cat(weights).contiguous()
    E = feat.shape[1]
    collect_s = time.time() - t0
    # training on the tensor cores
    trainer = qmc.QMC(prob.n, 1, seed, n_diag)
    trainer.load_schedule(prob)
    trainer.set_mlp(net)
    params = torch.tensor(TR.pack(net), device="cuda")
    mo, vo = torch.zeros_like(params), torch.zeros_like(params)
    torch.cuda.synchronize()
    t1 = time.time()
    losses = []
    for t in range(1, train_steps + 1):
        loss, grad = trainer.learn_grad_tc(params, feat, target_t, weight, E)
        losses.append(loss)
        trainer.learn_adam(params, grad, mo, vo, t, 3e-3)
    torch.cuda.synchronize()
    train_s = time.time() - t1
    trained = TR.unpack(params.cpu().numpy(), net)
    trainer.close()
    # comparison
    rows = []
    for rule, kind, netw in (("exact", qmc.PROPOSAL_EXACT, None), ("static", qmc.PROPOSAL_STATIC, None),
                             ("learned_tc_untrained", qmc.PROPOSAL_LEARNED_TC, net),
                             ("learned_tc_trained", qmc.PROPOSAL_LEARNED_TC, trained)):
        sim = qmc.QMC(prob.n, nvec, seed + 1, n_diag, integrator=qmc.AB2, initiator_min=init_min,
                      stream=torch.cuda.current_stream().cuda_stream)
        sim.load_schedule(prob)
        if netw is not None:
            sim.set_mlp(netw)
        sim.set_proposal(kind)
        sim.init_populations(rho0)
        torch.cuda.synchronize()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record()
        planner.run(sim, pl)
        ev1.record()
        torch.cuda.synchronize()
        sec = ev0.elapsed_time(ev1) * 1e-3
        fid = _final_fidelity(sim, target, n_diag)
        spread = float(fid.std(ddof=1))
        rows.append({"rule": rule, "fidelity": float(fid.mean()), "spread": spread, "seconds": sec,
                     "walkers_needed_1e-3": n_diag * (spread / 1e-3) ** 2,
                     "time_to_1e-3_s": sec * (spread / 1e-3) ** 2 / nvec})
        sim.close()
    return {"workload": name, "n": prob.n, "G": len(net["out_masks"]), "hidden": hidden, "events": E,
            "collect_s": collect_s, "train_steps": train_steps, "train_s": train_s,
            "loss_first": losses[0], "loss_last": losses[-1], "nvec": nvec, "n_diag": n_diag, "xi": xi,
            "t_end": t_end, "rules": rows}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("study", choices=["initiator", "replicas", "proposal"])
    ap.add_argument("--workload", default="ghz24")
    ap.add_argument("--events", type=int, default=10**7)
    ap.add_argument("--out", default=None)
    ap.add_argument("--sizes", default=None, help="comma-separated qubit counts")
    ap.add_argument("--state", default="plus", choices=["plus", "w"])
    ap.add_argument("--nvec", type=int, default=16)
    ap.add_argument("--n-diag", type=int, default=0)
    ap.add_argument("--xi", type=float, default=0.0)
    ap.add_argument("--replicas", type=int, default=5)
    ap.add_argument("--t-end", type=float, default=4.0,
                    help="replicas: end time (4.5 completes the DD cycle on both sublattices)")
    args = ap.parse_args()
    import torch
    torch.cuda.init()
    t0 = time.time()
    if args.study == "initiator":
        sizes = tuple(int(v) for v in args.sizes.split(",")) if args.sizes else (8, 16, 24, 32)
        res = {"rows": initiator_study(sizes, nvec=args.nvec, n_diag=args.n_diag or 10**5)}
    elif args.study == "replicas":
        sizes = tuple(int(v) for v in args.sizes.split(",")) if args.sizes else (8, 10, 12, 14)
        res = replica_study(sizes, state=args.state, n_diag=args.n_diag or 2 * 10**5, xi=args.xi,
                            replicas=args.replicas, t_end=args.t_end)
    else:
        res = proposal_study(args.workload, nvec=args.nvec, n_diag=args.n_diag or 10**5, train_events=args.events)
    res["wall_s"] = time.time() - t0
    txt = json.dumps(res, indent=1)
    if args.out:
        with open(args.out, "w") as f:
            f.write(txt)
    print(txt)


if __name__ == "__main__":
    main()
