"""Launch shapes and the autotuner (qmc_set_tuning, qmc_autotune): results
never depend on them.  Every draw is keyed by step, vector, key and walker and
the heavy and light spawn paths give the same spawns, so the populations are
bit-identical under extreme shapes (one CTA per kernel, every parent heavy or
none, 4 or 256 records per sort bucket), and a context that ran the autotuner
steps exactly like one that did not."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2502_18929_gb300 import problems as P
from paper_2502_18929_gb300 import qmc

pytestmark = pytest.mark.gpu


def _run(prob, tuning=None, autotune=False, steps=120):
    sim = qmc.QMC(prob.n, 6, 17, 20000)
    sim.load_schedule(prob)
    if tuning is not None:
        sim.set_tuning(**tuning)
    sim.init_populations(P.rho_basis(0))
    sim.step(0.01, 60)
    chosen = sim.autotune(0.01, 3) if autotune else None
    sim.step(0.01, steps)
    out = [sim.export(s) for s in range(sim.nseg)]
    obs = sim.observables()
    sim.close()
    return out, obs, chosen


def _same(a, b, where):
    for s, ((ka, ra, ia), (kb, rb, ib)) in enumerate(zip(a, b)):
        assert np.array_equal(ka, kb) and np.array_equal(ra, rb) and np.array_equal(ia, ib), f"{where} vector {s}"


@pytest.mark.parametrize("tuning", [
    {"max_ctas": 1, "heavy_walkers": 256, "bucket_records": 24},
    {"max_ctas": 0, "heavy_walkers": 16, "bucket_records": 4},
    {"max_ctas": 5, "heavy_walkers": 1 << 20, "bucket_records": 256},
])
def test_results_do_not_depend_on_launch_shapes(tuning):
    prob = P.ghz_circuit(5)
    ref, ref_obs, _ = _run(prob)
    got, got_obs, _ = _run(prob, tuning=tuning)
    _same(ref, got, str(tuning))
    assert np.array_equal(ref_obs, got_obs)


def test_autotune_keeps_the_state_and_picks_listed_shapes():
    prob = P.ghz_circuit(5)
    ref, ref_obs, _ = _run(prob)
    got, got_obs, chosen = _run(prob, autotune=True)
    _same(ref, got, "after autotune")
    assert np.array_equal(ref_obs, got_obs)
    assert chosen["heavy_walkers"] in (64, 256, 1024)
    assert chosen["bucket_records"] in (12, 24, 48)
    assert chosen["max_ctas"] >= 0


def test_autotune_then_oracle():
    prob = P.ghz_circuit(4)
    sim = qmc.QMC(4, 4, 5, 5000)
    sim.load_schedule(prob)
    sim.init_populations(P.rho_basis(0))
    sim.step(0.01, 30)
    sim.autotune(0.01, 2)
    sim.step(0.01, 70)
    orc = O.OracleSim(prob, 4, 5, integrator=qmc.AB2, n_diag=5000)
    orc.init(P.rho_basis(0))
    assert orc.step(0.01, 100) == O.OK
    for v in range(4):
        k, r, i = sim.export(v)
        ok, orr, oi = orc.population(v)
        assert np.array_equal(k, ok) and np.array_equal(r, orr) and np.array_equal(i, oi), v


def test_tuning_range_checked():
    sim = qmc.QMC(3, 1, 1, 100)
    with pytest.raises(qmc.QmcError):
        sim.set_tuning(heavy_walkers=8)
    with pytest.raises(qmc.QmcError):
        sim.set_tuning(bucket_records=1000)
    sim.set_tuning(max_ctas=3, heavy_walkers=64, bucket_records=12)
    assert sim.get_tuning() == {"max_ctas": 3, "heavy_walkers": 64, "bucket_records": 12}
