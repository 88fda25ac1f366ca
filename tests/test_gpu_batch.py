"""Batched step (qmc_batch_create): several problem instances of different
sizes and schedules share every launch of a step.  Each instance's vectors
must be bit-identical to the same instance run alone (same seed, same vector
count), and, for a few instances, to the oracle.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2502_18929_gb300 import problems as P
from paper_2502_18929_gb300 import qmc

pytestmark = pytest.mark.gpu


def _instances(k, seed):
    """GHZ circuits of 3..9 qubits with oscillating (non-Markovian) rates:
    gamma0 ~ U[0.01, 0.05], omega ~ U[0.5, 2], N^diag log-uniform."""
    rng = np.random.default_rng(seed)
    probs, nvec, seeds, ndiag, mins = [], [], [], [], []
    for i in range(k):
        n = int(rng.integers(3, 10))
        g0 = float(rng.uniform(0.01, 0.05))
        om = float(rng.uniform(0.5, 2.0))
        probs.append(P.ghz_circuit(n, gamma1=g0, gamma_phi=g0, rate_kind=P.RATE_COS, omega1=om, omega_phi=om))
        nvec.append(int(rng.integers(1, 4)))
        seeds.append(1000 + 17 * i)
        ndiag.append(int(10 ** rng.uniform(3.0, 3.8)))
        mins.append(0 if i % 3 else 2)
    return probs, nvec, seeds, ndiag, mins


def _export_all(sim, segs):
    return [sim.export(s) for s in segs]


def _same(a, b, where):
    for s, ((ka, ra, ia), (kb, rb, ib)) in enumerate(zip(a, b)):
        assert ka.size == kb.size, f"{where} vector {s}: {ka.size} vs {kb.size} records"
        assert np.array_equal(ka, kb) and np.array_equal(ra, rb) and np.array_equal(ia, ib), f"{where} vector {s}"


@pytest.mark.parametrize("max_ctas", [0, 3])
def test_batch_matches_instances_alone(max_ctas):
    probs, nvec, seeds, ndiag, mins = _instances(7, 5)
    batch = qmc.QMC.batch(probs, nvec, seeds, ndiag, initiator_mins=mins, max_ctas=max_ctas)
    batch.init_populations(P.rho_basis(0))
    for chunk in range(3):
        batch.step(0.01, 50)
    off = batch.offsets
    obs = batch.observables()
    for i, prob in enumerate(probs):
        alone = qmc.QMC(prob.n, nvec[i], seeds[i], ndiag[i], initiator_min=mins[i], max_ctas=max_ctas)
        alone.load_schedule(prob)
        alone.init_populations(P.rho_basis(0))
        for chunk in range(3):
            alone.step(0.01, 50)
        _same(_export_all(batch, range(off[i], off[i + 1])), _export_all(alone, range(nvec[i])), f"instance {i}")
        assert np.array_equal(obs[off[i]:off[i + 1]], alone.observables()), f"instance {i} observables"
        alone.close()
    assert batch.clock()[0] == 150


def test_batch_matches_oracle():
    probs, nvec, seeds, ndiag, mins = _instances(4, 9)
    batch = qmc.QMC.batch(probs, nvec, seeds, ndiag, initiator_mins=mins)
    batch.init_populations(P.rho_basis(0))
    batch.step(0.01, 120)
    off = batch.offsets
    for i in (0, 3):
        orc = O.OracleSim(probs[i], nvec[i], seeds[i], integrator=qmc.AB2, init_min=mins[i], n_diag=ndiag[i])
        orc.init(P.rho_basis(0))
        assert orc.step(0.01, 120) == O.OK
        for v in range(nvec[i]):
            k, r, im = batch.export(off[i] + v)
            ok, orr, oi = orc.population(v)
            assert np.array_equal(k, ok) and np.array_equal(r, orr) and np.array_equal(im, oi), f"inst {i} vec {v}"


def test_batch_rejects_load_schedule():
    probs, nvec, seeds, ndiag, mins = _instances(2, 3)
    batch = qmc.QMC.batch(probs, nvec, seeds, ndiag)
    with pytest.raises(qmc.QmcError):
        batch.load_schedule(probs[0])
