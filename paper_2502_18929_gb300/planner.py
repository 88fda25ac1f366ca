"""Step-size planning for a run over [t_start, t_end).

The walker method needs p < 1 for every spawn [End Matter, spawn step]; square
pulses of large amplitude (a pi pulse of width 0.02 has |h| ~ 78.5) need a
smaller step than the idle evolution.  The run is split at every pulse-window
edge; inside a piece the step is the largest dt' <= dt that divides the piece
evenly and keeps a bound on p below ``p_cap`` (AB2 factor 3/2 included).  A
change of step size restarts AB2 with one Euler step.

The bound is taken from the problem description only: every expanded term's
magnitude is at most 2 |h rate| per Hamiltonian term and 2 |gamma| (sum_a |l_a|)^2
per Lindblad operator, and |Re c| + |Im c| <= sqrt(2) |c|.
"""
from __future__ import annotations

import math

from .problems import Problem


def _rate(prob: Problem, rid: int, t: float) -> float:
    kind, a, b, c = prob.rates[rid]
    return abs(a) if kind == 0 else abs(a)  # |a cos(.)| <= |a|


def _on(prob: Problem, wid: int, t0: float, t1: float) -> bool:
    if wid < 0:
        return True
    w0, w1 = prob.windows[wid]
    return w0 < t1 and t0 < w1


def column_norm_bound(prob: Problem, t0: float, t1: float) -> float:
    """Upper bound of sum_kl (|Re L| + |Im L|) for any state on [t0, t1)."""
    acc = 0.0
    for h, xm, zm, rid, wid in prob.ham:
        if _on(prob, wid, t0, t1):
            acc += 2.0 * abs(h) * _rate(prob, rid, t0)
    for ops, rid, wid in prob.lind:
        if _on(prob, wid, t0, t1):
            s = sum(abs(c) for c, _, _ in ops)
            acc += 2.0 * _rate(prob, rid, t0) * s * s
    return math.sqrt(2.0) * acc


def plan(prob: Problem, t_end: float, dt: float, p_cap: float = 0.5, t_start: float = 0.0):
    """List of ``(t0, dt_piece, nsteps)`` covering [t_start, t_end)."""
    edges = sorted({e for e in prob.boundaries(t_end) if t_start <= e <= t_end} | {t_start, t_end})
    out = []
    for a, b in zip(edges[:-1], edges[1:]):
        length = b - a
        if length <= 0.0:
            continue
        bound = column_norm_bound(prob, a, b)
        dmax = dt if bound <= 0.0 else min(dt, p_cap / (1.5 * bound))
        n = max(1, int(math.ceil(length / dmax - 1e-9)))
        out.append((a, length / n, n))
    return out


def total_steps(pl) -> int:
    return sum(n for _, _, n in pl)


def run(sim, pl, max_steps: int | None = None) -> int:
    """Drive ``sim`` (library ``QMC`` or oracle ``OracleSim``) through a plan.
    Each piece starts by setting the clock time to its left edge (no drift).
    Returns the number of steps taken."""
    done = 0
    for t0, d, n in pl:
        if max_steps is not None:
            n = min(n, max_steps - done)
        if n <= 0:
            break
        step, _, tp, dl, pv = sim.clock()
        sim.set_clock(step, t0, tp, dl, pv)
        rc = sim.step(d, n)
        if rc not in (None, 0):
            raise RuntimeError(f"step failed with code {rc}")
        done += n
    return done
