"""The Redfield two-qubit model (Eq. (4); End Matter on the Redfield equation)
as a problem description, and the oracle's walker dynamics on it.

* Pins of the description: the dissipator rates against the values the paper
  prints (tests/golden/redfield_rates.txt) and its closed form; the dense
  Liouvillian of the Pauli-sum problem against the Redfield superoperator
  built directly from the frequency matrix A and the rate matrix over the jump
  operators s_1^-, s_2^-, moved to the paper's Lindblad-operator basis; trace
  preservation.
* The walker method on it (negative rate: non-Markovian): the mean of the
  tracked populations rho~_00, rho~_11, rho~_22 over vectors equals the dense
  AB2 recursion (each within the family-wise bound of three observables).
"""
import math
import os

import numpy as np

from oracle import dense as Dn
from oracle import oracle as O
from paper_2502_18929_gb300 import planner
from paper_2502_18929_gb300 import problems as P
from stat_bounds import familywise

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "redfield_rates.txt")


def _golden():
    rows = [ln.split() for ln in open(GOLDEN) if ln.strip() and not ln.startswith("#")]
    return [[float(v) for v in r] for r in rows]


def test_rates_match_the_paper():
    for w1, w2, g1, g2, a, k, l1, l2 in _golden():
        _, info = P.redfield_two_qubits(w1, w2, g1, g2, a, k)
        lam = sorted(info["lam"])
        assert round(lam[0], 4) == l1 and round(lam[1], 4) == l2
        root = math.sqrt((g1 * g1 + g2 * g2 + 8 * k * k) / 8)
        assert abs(lam[0] - ((g1 + g2) / 4 - root)) < 1e-12
        assert abs(lam[1] - ((g1 + g2) / 4 + root)) < 1e-12


def _lowering(q):
    """s_q^- on two qubits (qubit q is bit q), built entry by entry."""
    m = np.zeros((4, 4), dtype=np.complex128)
    for x in range(4):
        if (x >> q) & 1:
            m[x ^ (1 << q), x] = 1.0
    return m


def _superop(H, terms):
    """Column-vectorised -i[H, .] + sum c (A . B^dag - {B^dag A, .}/2)."""
    I = np.eye(4)
    L = -1j * np.kron(I, H) + 1j * np.kron(H.T, I)
    for c, A, B in terms:
        BdA = B.conj().T @ A
        L += c * (np.kron(B.conj(), A) - 0.5 * np.kron(I, BdA) - 0.5 * np.kron(BdA.T, I))
    return L


def test_liouvillian_equals_the_redfield_superoperator():
    for args in ((0.25, 0.5, 1.0, 4.0, 3.0, 1.0), (0.7, 0.2, 2.5, 0.5, -1.0, 0.4)):
        prob, info = P.redfield_two_qubits(*args)
        A, G, V = info["A"], info["G"], info["V"]
        s = [_lowering(0), _lowering(1)]
        H = sum(A[i, j] * s[j].conj().T @ s[i] for i in range(2) for j in range(2))
        direct = _superop(H, [(G[i, j], s[j], s[i]) for i in range(2) for j in range(2)])
        # rho~ = V^dag rho V, so vec(rho~) = (V^T kron V^dag) vec(rho)
        T = np.kron(V.T, V.conj().T)
        moved = T @ direct @ np.linalg.inv(T)
        assert np.abs(Dn.liouvillian(prob, 0.0) - moved).max() < 1e-12
        # trace preservation: vec(I)^T L = 0
        assert np.abs(Dn.vec(np.eye(4)) @ Dn.liouvillian(prob, 0.0)).max() < 1e-12


def rho0():
    return P.rho_pure({0: 1.0, 1: 1.0, 2: 1.0})


def test_walkers_match_dense_ab2():
    prob, _ = P.redfield_two_qubits()
    pl = planner.plan(prob, 2.0, 0.005)
    V, nd = 16, 20000
    sim = O.OracleSim(prob, V, seed=3, integrator=O.AB2, n_diag=nd)
    sim.init(rho0())
    planner.run(sim, pl)
    rhos = np.array([sim.density(s) / nd for s in range(V)])
    steps = planner.total_steps(pl)
    assert len(pl) == 1
    ref = Dn.evolve(prob, Dn.rho_from_entries(2, rho0()), pl[0][1], steps, "ab2")
    thr = familywise(3, V)
    for b in range(3):
        vals = rhos[:, b, b].real
        se = vals.std(ddof=1) / math.sqrt(V)
        assert abs(vals.mean() - ref[b, b].real) < thr * se, (b, vals.mean(), ref[b, b].real, se)
