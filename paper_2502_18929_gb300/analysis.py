"""Host-side estimators over the per-vector results the library returns.

None of this is on the step's path; it turns exact per-vector integers
(N^diag, overlaps, anti-Hermiticity, occupied-state counts) into the paper's
reported quantities.

* Replica aggregation [Markovian circuit dynamics, replica paragraph]:
  r independent replicas of N^diag walkers each form one estimator with
  N^diag_eff = r N^diag; rho_QMC = sum_j N^(j) / N^diag_eff, its trace
  sum_j N^diag_j(t) / N^diag_eff, a fidelity |sum_j <psi|N^(j)|psi>| /
  N^diag_eff.
* Error bars: 95 % confidence intervals by bootstrapping over the independent
  samples [End Matter, simulation methodology].
* The subspace-size model dim(H_QMC) = C e^(beta n) (N^diag)^gamma and the
  anti-Hermiticity model eps = A e^(alpha n) (N^diag)^(-1/2) + eps_inf, fitted
  by least squares [Markovian circuit dynamics; End Matter on Hermiticity
  preservation], and the walker number N^diag_opt(n, tau) that the second
  one predicts for a tolerance tau.
"""
from __future__ import annotations

import math

import numpy as np


def aggregate(values, n_diag: int) -> dict:
    """Replica aggregate of per-replica sums: ``values`` holds, per replica j,
    a quantity linear in N^(j) (N^diag_j, an overlap <psi|N^(j)|psi>, ...);
    returns the aggregate estimate sum_j values_j / (r N^diag) and N^diag_eff."""
    v = np.asarray(values)
    r = v.shape[0]
    return {"n_diag_eff": r * int(n_diag), "estimate": v.sum(axis=0) / (r * float(n_diag)),
            "per_replica": v / float(n_diag)}


def bootstrap_ci(samples, stat=np.mean, n_boot: int = 10000, level: float = 0.95, seed: int = 0):
    """Percentile bootstrap interval of ``stat`` over independent samples
    (axis 0): (estimate, low, high)."""
    x = np.asarray(samples, dtype=np.float64)
    rng = np.random.default_rng(seed)
    idx = rng.integers(0, x.shape[0], size=(n_boot, x.shape[0]))
    boots = np.array([stat(x[i]) for i in idx])
    lo, hi = np.quantile(boots, [(1.0 - level) / 2.0, (1.0 + level) / 2.0], axis=0)
    return stat(x), lo, hi


def fit_subspace(n, n_diag, dim) -> dict:
    """Least squares of log dim = log C + beta n + gamma log N^diag."""
    n = np.asarray(n, dtype=np.float64)
    nd = np.asarray(n_diag, dtype=np.float64)
    y = np.log(np.asarray(dim, dtype=np.float64))
    M = np.stack([np.ones_like(n), n, np.log(nd)], axis=1)
    coef, *_ = np.linalg.lstsq(M, y, rcond=None)
    return {"C": float(math.exp(coef[0])), "beta": float(coef[1]), "gamma": float(coef[2]),
            "rms_log": float(np.sqrt(np.mean((M @ coef - y) ** 2)))}


def fit_antiherm(n, n_diag, eps, alphas=None) -> dict:
    """eps = A e^(alpha n) / sqrt(N^diag) + eps_inf: for each alpha on a grid
    (refined around the best) A and eps_inf by linear least squares; returns
    the (alpha, A, eps_inf) with the smallest squared residual."""
    n = np.asarray(n, dtype=np.float64)
    nd = np.asarray(n_diag, dtype=np.float64)
    y = np.asarray(eps, dtype=np.float64)

    def solve(a):
        M = np.stack([np.exp(a * n) / np.sqrt(nd), np.ones_like(n)], axis=1)
        c, *_ = np.linalg.lstsq(M, y, rcond=None)
        return float(np.sum((M @ c - y) ** 2)), c

    grid = np.linspace(-1.0, 1.0, 401) if alphas is None else np.asarray(alphas, dtype=np.float64)
    best = min(grid, key=lambda a: solve(a)[0])
    step = grid[1] - grid[0] if len(grid) > 1 else 0.01
    # golden-section refinement inside the grid cell pair around the optimum
    lo, hi = best - step, best + step
    g = (math.sqrt(5.0) - 1.0) / 2.0
    a1, a2 = hi - g * (hi - lo), lo + g * (hi - lo)
    f1, f2 = solve(a1)[0], solve(a2)[0]
    for _ in range(80):
        if f1 < f2:
            hi, a2, f2 = a2, a1, f1
            a1 = hi - g * (hi - lo)
            f1 = solve(a1)[0]
        else:
            lo, a1, f1 = a1, a2, f2
            a2 = lo + g * (hi - lo)
            f2 = solve(a2)[0]
    best = (lo + hi) / 2.0
    res, c = solve(best)
    return {"alpha": float(best), "A": float(c[0]), "eps_inf": float(c[1]), "sse": res}


def n_diag_opt(n: float, tau: float, fit: dict) -> float:
    """Smallest N^diag with A e^(alpha n) / sqrt(N^diag) + eps_inf <= tau
    (inf when tau <= eps_inf)."""
    room = tau - fit["eps_inf"]
    if room <= 0.0:
        return math.inf
    return (fit["A"] * math.exp(fit["alpha"] * n) / room) ** 2


def antiherm_epsilon(frob2, n_diag_eff: int) -> float:
    """epsilon = ||rho - rho^dagger||_F from the exact ||N - N^dagger||_F^2 of
    an (aggregated) population with N^diag_eff walkers on the diagonal."""
    return math.sqrt(float(frob2)) / float(n_diag_eff)
