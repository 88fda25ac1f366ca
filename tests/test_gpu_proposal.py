"""Static-weight proposal spawning on the GPU (qmc_set_proposal), bit-exact
against the oracle's proposal mode: heavy parents (GHZ-4 from |0><0|), light
parents of every walker-pair layout (n = 32 spread states in a CNOT window),
the DD ring, and a batch of instances."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2502_18929_gb300 import problems as P
from paper_2502_18929_gb300 import qmc

pytestmark = pytest.mark.gpu

STATIC = 1


def _pair(prob, nseg, seed, n_diag, integrator=qmc.AB2):
    gpu = qmc.QMC(prob.n, nseg, seed, n_diag, integrator=integrator)
    gpu.load_schedule(prob)
    gpu.set_proposal(STATIC)
    orc = O.OracleSim(prob, nseg, seed, integrator=integrator, n_diag=n_diag)
    orc.set_proposal(STATIC)
    return gpu, orc


def _same(gpu, orc, where):
    for s in range(gpu.nseg):
        gk, gr, gi = gpu.export(s)
        ok, orr, oi = orc.population(s)
        assert gk.size == ok.size, f"{where} vector {s}: {gk.size} vs {ok.size} records"
        assert np.array_equal(gk, ok) and np.array_equal(gr, orr) and np.array_equal(gi, oi), f"{where} vector {s}"


def test_static_proposal_ghz4_heavy_and_light():
    prob = P.ghz_circuit(4)
    gpu, orc = _pair(prob, 8, 3, 10000)
    gpu.init_populations(P.rho_basis(0))
    orc.init(P.rho_basis(0))
    for k in range(4):
        gpu.step(0.01, 100)
        assert orc.step(0.01, 100) == O.OK
        _same(gpu, orc, f"ghz4 chunk {k}")


def _spread(n, nseg, count, seed):
    return [P.spread_population(n, count + 37 * s, seed + s) for s in range(nseg)]


def test_static_proposal_spread_n32():
    prob = P.ghz_circuit(32)
    gpu, orc = _pair(prob, 2, 5, 10**6)
    cur, prev = _spread(32, 2, 12000, 7), _spread(32, 2, 11000, 70)
    gpu.set_populations(cur, which=0)
    gpu.set_populations(prev, which=1)
    gpu.set_clock(1234, 5.5, 5.49, 0.01, True)
    for s, (k, r, i) in enumerate(cur):
        orc.set_population(s, k, r, i, which=0)
    for s, (k, r, i) in enumerate(prev):
        orc.set_population(s, k, r, i, which=1)
    orc.set_clock(1234, 5.5, 5.49, 0.01, True)
    for k in range(3):
        gpu.step(0.01, 1)
        assert orc.step(0.01, 1) == O.OK
        _same(gpu, orc, f"n32 step {k}")


def test_static_proposal_dd_ring():
    prob = P.dd_ring(12, seed=5, t_end=3.0)
    gpu, orc = _pair(prob, 3, 77, 100000)
    cur, prev = _spread(12, 3, 20000, 1), _spread(12, 3, 19000, 50)
    gpu.set_populations(cur, which=0)
    gpu.set_populations(prev, which=1)
    gpu.set_clock(500, 0.2, 0.195, 0.005, True)
    for s, (k, r, i) in enumerate(cur):
        orc.set_population(s, k, r, i, which=0)
    for s, (k, r, i) in enumerate(prev):
        orc.set_population(s, k, r, i, which=1)
    orc.set_clock(500, 0.2, 0.195, 0.005, True)
    for k in range(3):
        gpu.step(0.005, 1)
        assert orc.step(0.005, 1) == O.OK
        _same(gpu, orc, f"dd step {k}")


def test_static_proposal_in_a_batch():
    probs = [P.ghz_circuit(n) for n in (3, 5, 4)]
    nvec, seeds, ndiag = [2, 1, 2], [11, 12, 13], [3000, 5000, 2000]
    batch = qmc.QMC.batch(probs, nvec, seeds, ndiag)
    batch.set_proposal(STATIC)
    batch.init_populations(P.rho_basis(0))
    batch.step(0.01, 160)
    off = batch.offsets
    for i, prob in enumerate(probs):
        orc = O.OracleSim(prob, nvec[i], seeds[i], integrator=qmc.AB2, n_diag=ndiag[i])
        orc.set_proposal(STATIC)
        orc.init(P.rho_basis(0))
        assert orc.step(0.01, 160) == O.OK
        for v in range(nvec[i]):
            k, r, im = batch.export(off[i] + v)
            ok, orr, oi = orc.population(v)
            assert np.array_equal(k, ok) and np.array_equal(r, orr) and np.array_equal(im, oi), f"inst {i} vec {v}"


def test_proposal_kind_checked():
    gpu = qmc.QMC(3, 1, 1, 100)
    with pytest.raises(qmc.QmcError):
        gpu.set_proposal(7)
