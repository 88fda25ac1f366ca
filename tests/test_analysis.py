"""Host-side estimators: replica aggregation, bootstrap intervals and the
paper's two empirical fits, checked on synthetic data with known answers."""
import math

import numpy as np

from paper_2502_18929_gb300 import analysis as A


def test_aggregate_is_the_pooled_estimate():
    vals = np.array([199_000, 201_500, 200_200, 199_900, 200_400])
    out = A.aggregate(vals, 200_000)
    assert out["n_diag_eff"] == 1_000_000
    assert out["estimate"] == vals.sum() / 1e6
    assert np.allclose(out["per_replica"], vals / 2e5)


def test_bootstrap_interval_covers_the_mean():
    rng = np.random.default_rng(7)
    hits = 0
    trials = 200
    for _ in range(trials):
        x = rng.normal(3.0, 2.0, size=40)
        est, lo, hi = A.bootstrap_ci(x, n_boot=2000, seed=int(rng.integers(1 << 30)))
        assert lo <= est <= hi
        hits += lo <= 3.0 <= hi
    # a 95 % interval: coverage of 200 trials within 3 binomial sigma of 0.95 (percentile
    # intervals run slightly narrow at n = 40)
    assert abs(hits / trials - 0.95) < 3 * math.sqrt(0.95 * 0.05 / trials) + 0.02


def test_subspace_fit_recovers_parameters():
    n = np.repeat([10, 12, 14, 16], 4)
    nd = np.tile([4e5, 6e5, 8e5, 1e6], 4)
    C, beta, gamma = 3.7, 0.208, 0.721
    dim = C * np.exp(beta * n) * nd ** gamma
    fit = A.fit_subspace(n, nd, dim)
    assert abs(fit["beta"] - beta) < 1e-10 and abs(fit["gamma"] - gamma) < 1e-10
    assert abs(fit["C"] / C - 1) < 1e-9


def test_antiherm_fit_and_optimal_walkers():
    n = np.repeat([10, 14, 18, 22], 4)
    nd = np.tile([4e5, 6e5, 8e5, 1e6], 4)
    Aa, alpha, einf = 1.3, 0.0715, 2e-4
    eps = Aa * np.exp(alpha * n) / np.sqrt(nd) + einf
    fit = A.fit_antiherm(n, nd, eps)
    assert abs(fit["alpha"] - alpha) < 1e-6 and abs(fit["A"] / Aa - 1) < 1e-5 and abs(fit["eps_inf"] - einf) < 1e-8
    nopt = A.n_diag_opt(20, 0.02, fit)
    assert abs(Aa * math.exp(alpha * 20) / math.sqrt(nopt) + einf - 0.02) < 1e-9
    assert A.n_diag_opt(20, 1e-4, fit) == math.inf


def test_epsilon_from_exact_norm():
    assert A.antiherm_epsilon(4 * 10**12, 10**6) == 2.0
