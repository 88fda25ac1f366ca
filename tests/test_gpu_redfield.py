"""The Redfield two-qubit model (Eq. (4), one negative rate) on the GPU.

* Parity: populations bit-identical to the oracle's after every checked step.
* The QMC side of Fig. 3: vectors of 10^6 walkers from (|0~> + |1~> +
  |2~>)/sqrt(3); the tracked populations rho~_00, rho~_11, rho~_22 and the
  trace N^diag(t) / N^diag(0), averaged over the vectors, follow the dense AB2
  recursion (family-wise bound over all checked times and observables), and
  a single vector stays within 0.02 of it.
"""
import math

import numpy as np
import pytest

from oracle import dense as Dn
from oracle import oracle as O
from paper_2502_18929_gb300 import planner
from paper_2502_18929_gb300 import problems as P
from paper_2502_18929_gb300 import qmc
from stat_bounds import familywise

pytestmark = pytest.mark.gpu


def rho0():
    return P.rho_pure({0: 1.0, 1: 1.0, 2: 1.0})


def test_redfield_parity():
    prob, _ = P.redfield_two_qubits()
    pl = planner.plan(prob, 1.0, 0.005)
    gpu = qmc.QMC(2, 6, 11, 5000)
    gpu.load_schedule(prob)
    orc = O.OracleSim(prob, 6, 11, integrator=O.AB2, n_diag=5000)
    gpu.init_populations(rho0())
    orc.init(rho0())
    for chunk in range(4):
        piece = [(pl[0][0] + chunk * 50 * pl[0][1], pl[0][1], 50)]
        planner.run(gpu, piece)
        planner.run(orc, piece)
        for s in range(6):
            for a, b in zip(gpu.export(s), orc.population(s)):
                assert np.array_equal(a, b), (chunk, s)


def test_redfield_walkers_follow_exact_dynamics():
    prob, _ = P.redfield_two_qubits()
    V, nd, dt = 8, 10**6, 0.005
    gpu = qmc.QMC(2, V, 5, nd)
    gpu.load_schedule(prob)
    gpu.init_populations(rho0())
    record = {}
    ref = Dn.evolve(prob, Dn.rho_from_entries(2, rho0()), dt, 400, "ab2",
                    record=lambda k, r: record.__setitem__(k + 1, r.copy()))
    assert ref is not None
    checks = list(range(50, 401, 50))
    thr = familywise(4 * len(checks), V)
    done = 0
    for k in checks:
        gpu.step(dt, k - done)
        done = k
        rho = np.zeros((V, 4), dtype=np.float64)
        trace = np.zeros(V)
        for s in range(V):
            keys, re, im = gpu.export(s)
            for key, a in zip(keys.tolist(), re.tolist()):
                x, y = key >> 2, key & 3
                if x == y:
                    rho[s, x] += a / nd
            trace[s] = rho[s].sum()
        exact = record[k]
        for b in range(3):
            vals = rho[:, b]
            se = vals.std(ddof=1) / math.sqrt(V)
            assert abs(vals.mean() - exact[b, b].real) < thr * se, (k, b)
            assert np.abs(vals - exact[b, b].real).max() < 0.02, (k, b)
        se = trace.std(ddof=1) / math.sqrt(V)
        assert abs(trace.mean() - 1.0) < thr * se + 1e-12, k
