"""Learned-proposal spawning on the GPU (qmc_set_proposal_mlp), bit-exact
against the oracle's learned mode: the network's destination weights, the
walker's slot draw and the floor + Bernoulli walker counts, for heavy
parents (GHZ-4 from |0><0|), light parents of every walker-pair layout
(n = 32 spread states, widest hidden layer, small static share so that
counts above one occur), a time-dependent schedule (DD ring), and a network
that leaves some destinations without an output."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2502_18929_gb300 import problems as P
from paper_2502_18929_gb300 import qmc

pytestmark = pytest.mark.gpu

LEARNED = qmc.PROPOSAL_LEARNED


def _pair(prob, nseg, seed, n_diag, net, integrator=qmc.AB2):
    gpu = qmc.QMC(prob.n, nseg, seed, n_diag, integrator=integrator)
    gpu.load_schedule(prob)
    gpu.set_mlp(net)
    gpu.set_proposal(LEARNED)
    orc = O.OracleSim(prob, nseg, seed, integrator=integrator, n_diag=n_diag)
    orc.set_mlp(net)
    orc.set_proposal(LEARNED)
    return gpu, orc


def _same(gpu, orc, where):
    for s in range(gpu.nseg):
        gk, gr, gi = gpu.export(s)
        ok, orr, oi = orc.population(s)
        assert gk.size == ok.size, f"{where} vector {s}: {gk.size} vs {ok.size} records"
        assert np.array_equal(gk, ok) and np.array_equal(gr, orr) and np.array_equal(gi, oi), f"{where} vector {s}"


def _spread(n, nseg, count, seed):
    return [P.spread_population(n, count + 37 * s, seed + s) for s in range(nseg)]


def _set_both(gpu, orc, cur, prev, clock):
    gpu.set_populations(cur, which=0)
    gpu.set_populations(prev, which=1)
    gpu.set_clock(*clock)
    for s, (k, r, i) in enumerate(cur):
        orc.set_population(s, k, r, i, which=0)
    for s, (k, r, i) in enumerate(prev):
        orc.set_population(s, k, r, i, which=1)
    orc.set_clock(*clock)


def test_learned_ghz4_heavy_and_light():
    prob = P.ghz_circuit(4)
    net = P.random_network(prob, hidden=16, seed=3, eps=0.25, scale=2.0)
    gpu, orc = _pair(prob, 8, 3, 10000, net)
    gpu.init_populations(P.rho_basis(0))
    orc.init(P.rho_basis(0))
    for k in range(4):
        gpu.step(0.01, 100)
        assert orc.step(0.01, 100) == O.OK
        _same(gpu, orc, f"ghz4 chunk {k}")


def test_learned_spread_n32_wide_net():
    prob = P.ghz_circuit(32)
    net = P.random_network(prob, hidden=64, seed=8, eps=0.05, scale=3.0)
    gpu, orc = _pair(prob, 2, 5, 10**6, net)
    _set_both(gpu, orc, _spread(32, 2, 12000, 7), _spread(32, 2, 11000, 70), (1234, 5.5, 5.49, 0.01, True))
    for k in range(3):
        gpu.step(0.01, 1)
        assert orc.step(0.01, 1) == O.OK
        _same(gpu, orc, f"n32 step {k}")


def test_learned_dd_ring_partial_outputs():
    prob = P.dd_ring(12, seed=5, t_end=3.0)
    net = P.random_network(prob, hidden=24, seed=2, eps=0.1, scale=2.5)
    keep = np.arange(len(net["out_masks"])) % 3 != 1   # some destinations get no output
    for k in ("out_masks", "w3", "b3"):
        net[k] = net[k][keep]
    gpu, orc = _pair(prob, 3, 77, 100000, net)
    _set_both(gpu, orc, _spread(12, 3, 20000, 1), _spread(12, 3, 19000, 50), (500, 0.2, 0.195, 0.005, True))
    for k in range(3):
        gpu.step(0.005, 1)
        assert orc.step(0.005, 1) == O.OK
        _same(gpu, orc, f"dd step {k}")


def test_learned_euler_steps_ghz5():
    prob = P.ghz_circuit(5)
    net = P.random_network(prob, hidden=8, seed=11, eps=0.5, scale=1.0)
    gpu, orc = _pair(prob, 4, 19, 3000, net, integrator=qmc.EULER)
    gpu.init_populations(P.rho_basis(0))
    orc.init(P.rho_basis(0))
    gpu.step(0.02, 150)
    assert orc.step(0.02, 150) == O.OK
    _same(gpu, orc, "ghz5 euler")


def test_learned_refusals():
    prob = P.ghz_circuit(3)
    gpu = qmc.QMC(3, 1, 1, 100)
    gpu.load_schedule(prob)
    with pytest.raises(qmc.QmcError):
        gpu.set_proposal(LEARNED)          # no network loaded
    bad = P.random_network(P.ghz_circuit(4), hidden=4)
    with pytest.raises(qmc.QmcError):
        gpu.set_mlp(bad)                   # n_in = 9 for 3 qubits
    wide = P.random_network(prob, hidden=65)
    with pytest.raises(qmc.QmcError):
        gpu.set_mlp(wide)                  # hidden width above 64
    rep = P.random_network(prob, hidden=4)
    rep["out_masks"] = np.repeat(rep["out_masks"][:1], len(rep["out_masks"]))
    with pytest.raises(qmc.QmcError):
        gpu.set_mlp(rep)                   # repeated output masks
    batch = qmc.QMC.batch([prob, prob], [1, 1], [1, 2], [100, 100])
    with pytest.raises(qmc.QmcError):
        batch.set_mlp(P.random_network(prob, hidden=4))
