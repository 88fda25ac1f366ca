"""Pins of the oracle's proposal spawning (the library's alternative to the
exact |L|-weighted destination choice; not in the paper).

A walker attempts with p_att = sum of the destinations' static weights, picks
a destination in proportion to its static weight, and spawns onto the Re or
Im channel with the exact element weights inside that interval.  Each
destination and channel then receives w / 2^52 spawns per walker in
expectation, as in the plain method, so:

* the mean population follows the same deterministic Euler / AB2 recursion
  as the plain method [End Matter, simulation methodology];
* a one-step average over many vectors matches (I + dt L) N exactly (this
  fails if a static weight were below |Re L| + |Im L| of its destination,
  or a destination or channel were dropped).
"""
import numpy as np

from oracle import dense as Dn
from oracle import oracle as O
from paper_2502_18929_gb300 import problems as P
from stat_bounds import familywise


def _densities(prob, rho0, V, seed, dt, nsteps, proposal, integrator=O.AB2, n_diag=10000, net=None):
    sim = O.OracleSim(prob, V, seed=seed, integrator=integrator, n_diag=n_diag)
    if net is not None:
        sim.set_mlp(net)
    sim.set_proposal(proposal)
    sim.init(rho0)
    assert sim.step(dt, nsteps) == O.OK
    return np.array([sim.density(s) / n_diag for s in range(V)])


def test_static_proposal_exact_mean_ghz4_ab2():
    """GHZ-4 preparation, 16 vectors x 1e4 walkers, 400 AB2 steps, proposal
    spawning: the mean density equals the dense AB2 recursion."""
    prob = P.ghz_circuit(4)
    rho0 = P.rho_basis(0)
    rhos = _densities(prob, rho0, 16, 21, 0.01, 400, proposal=1)
    ref = Dn.evolve(prob, Dn.rho_from_entries(4, rho0), 0.01, 400, "ab2")
    se = rhos.std(0, ddof=1) / np.sqrt(rhos.shape[0])
    sig = np.abs(ref) > 0.01
    z = np.abs(rhos.mean(0) - ref)[sig] / se[sig]
    assert z.max() < familywise(2 * sig.sum(), rhos.shape[0]), z.max()


def test_static_proposal_one_step_mean():
    """One Euler step from a mixed state of a 3-qubit noisy circuit inside a
    CNOT window: the average over 400 vectors of N(t + dt) equals
    (I + dt L) N(t) within sampling error."""
    prob = P.ghz_circuit(3)
    rho0 = [(0, 0, 0.5, 0.0), (1, 1, 0.25, 0.0), (0, 1, 0.2, 0.1), (1, 0, 0.2, -0.1), (3, 3, 0.25, 0.0)]
    V = 400
    sim = O.OracleSim(prob, V, seed=5, integrator=O.EULER, n_diag=4000)
    sim.set_proposal(1)
    sim.init(rho0)
    n0 = np.array([sim.density(s) for s in range(V)])
    sim.set_clock(250, 2.5)
    assert sim.step(0.05, 1) == O.OK
    n1 = np.array([sim.density(s) for s in range(V)])
    Lm = Dn.liouvillian(prob, 2.5)
    d = 8
    pred = np.array([Dn.unvec((np.eye(d * d) + 0.05 * Lm) @ Dn.vec(r), d) for r in n0])
    diff = n1 - pred
    se = diff.std(0, ddof=1) / np.sqrt(V) + 1e-9
    z = np.abs(diff.mean(0)) / se
    assert z.max() < familywise(2 * diff[0].size, V), z.max()


def test_static_proposal_differs_from_plain_draws():
    """Same seeds, different choice rule: the populations differ (the mode
    is really switched), while both stay unbiased (tests above)."""
    prob = P.ghz_circuit(4)
    a = _densities(prob, P.rho_basis(0), 2, 7, 0.01, 150, proposal=0)
    b = _densities(prob, P.rho_basis(0), 2, 7, 0.01, 150, proposal=1)
    assert not np.allclose(a, b)


def test_learned_proposal_exact_mean_ghz4_ab2():
    """Learned proposal with an untrained (random) network mixed with 25 %
    static proposal: still unbiased, the mean equals the dense AB2 recursion
    (any q whose support covers the column's is unbiased)."""
    prob = P.ghz_circuit(4)
    rho0 = P.rho_basis(0)
    net = P.random_network(prob, hidden=16, seed=3, eps=0.25, scale=2.0)
    rhos = _densities(prob, rho0, 16, 31, 0.01, 400, proposal=2, net=net)
    ref = Dn.evolve(prob, Dn.rho_from_entries(4, rho0), 0.01, 400, "ab2")
    se = rhos.std(0, ddof=1) / np.sqrt(rhos.shape[0])
    sig = np.abs(ref) > 0.01
    z = np.abs(rhos.mean(0) - ref)[sig] / se[sig]
    assert z.max() < familywise(2 * sig.sum(), rhos.shape[0]), z.max()


def test_learned_proposal_one_step_mean():
    """One Euler step with a random network and a small static share (5 %),
    where amplitudes above 1 occur: the 400-vector mean matches (I + dt L) N."""
    prob = P.ghz_circuit(3)
    rho0 = [(0, 0, 0.5, 0.0), (1, 1, 0.25, 0.0), (0, 1, 0.2, 0.1), (1, 0, 0.2, -0.1), (3, 3, 0.25, 0.0)]
    V = 400
    sim = O.OracleSim(prob, V, seed=9, integrator=O.EULER, n_diag=4000)
    sim.set_mlp(P.random_network(prob, hidden=8, seed=4, eps=0.05, scale=3.0))
    sim.set_proposal(2)
    sim.init(rho0)
    n0 = np.array([sim.density(s) for s in range(V)])
    sim.set_clock(250, 2.5)
    assert sim.step(0.05, 1) == O.OK
    n1 = np.array([sim.density(s) for s in range(V)])
    Lm = Dn.liouvillian(prob, 2.5)
    pred = np.array([Dn.unvec((np.eye(64) + 0.05 * Lm) @ Dn.vec(r), 8) for r in n0])
    diff = n1 - pred
    se = diff.std(0, ddof=1) / np.sqrt(V) + 1e-9
    z = np.abs(diff.mean(0)) / se
    assert z.max() < familywise(2 * diff[0].size, V), z.max()


def test_learned_proposal_with_an_empty_column():
    """After the only pulse has ended no term is active: the static column is
    empty, nothing attempts and the population stays as it was (the learned
    weights of an empty column are never indexed)."""
    prob = P.Problem(n=2, name="h-pulse")
    P.add_hadamard_pulse(prob, 0, 0.0, 1.0)
    sim = O.OracleSim(prob, 2, seed=3, integrator=O.EULER, n_diag=500)
    sim.set_mlp(P.random_network(prob, hidden=4, seed=1, eps=0.5))
    sim.set_proposal(2)
    sim.init([(0, 0, 0.6, 0.0), (1, 1, 0.4, 0.0), (0, 1, 0.2, 0.1)])
    before = [sim.population(s) for s in range(2)]
    sim.set_clock(150, 1.5)
    assert sim.step(0.01, 5) == O.OK
    for s in range(2):
        k0, r0, i0 = before[s]
        k1, r1, i1 = sim.population(s)
        assert np.array_equal(k0, k1) and np.array_equal(r0, r1) and np.array_equal(i0, i1)
