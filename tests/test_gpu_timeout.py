"""Failure path of the bounded device waits (no GPU fault involved).

With a spin limit of 0 every wait on another CTA's look-back word gives up at
its first poll.  A step whose merge spans several tiles then stops with
QMC_ERR_DEVICE_TIMEOUT and names the wait site; the context keeps the
populations of the last completed step, and once the limit is restored the
next call repeats the failed step and matches the oracle bit for bit.  Every
kernel returns on its own: nothing waits without a limit.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2502_18929_gb300 import problems as P
from paper_2502_18929_gb300 import qmc

pytestmark = pytest.mark.gpu


def _state(n, nseg, count, seed):
    return [P.spread_population(n, count + 37 * s, seed + s) for s in range(nseg)]


def _same(gpu, orc, which, where):
    for s in range(gpu.nseg):
        for a, b in zip(gpu.export(s, which), orc.population(s, which)):
            assert np.array_equal(a, b), f"{where}: vector {s} differs"


@pytest.mark.parametrize("max_ctas", [0, 3])
def test_lookback_timeout_keeps_state_and_recovers(max_ctas):
    prob = P.ghz_circuit(32)
    nseg, seed, dt = 2, 23, 0.01
    gpu = qmc.QMC(32, nseg, seed, 10**6, integrator=qmc.AB2, max_ctas=max_ctas)
    gpu.load_schedule(prob)
    orc = O.OracleSim(prob, nseg, seed, integrator=O.AB2, n_diag=10**6)
    cur, prev = _state(32, nseg, 15000, 3), _state(32, nseg, 14000, 40)
    gpu.set_populations(cur, which=0)
    gpu.set_populations(prev, which=1)
    for s in range(nseg):
        orc.set_population(s, *cur[s], which=0)
        orc.set_population(s, *prev[s], which=1)
    gpu.set_clock(700, 5.2, 5.2 - dt, dt, True)
    orc.set_clock(700, 5.2, 5.2 - dt, dt, True)

    gpu.step(dt, 2)
    assert orc.step(dt, 2) == O.OK
    _same(gpu, orc, 0, "before")
    clock = gpu.clock()

    gpu.set_spin_limit(0)
    with pytest.raises(qmc.QmcError) as ei:
        gpu.step(dt, 3)
    assert ei.value.code == qmc.ERR_DEVICE_TIMEOUT
    assert "wait site" in str(ei.value)
    # the state of the last completed step: both population slots and the clock
    assert gpu.clock() == clock
    _same(gpu, orc, 0, "after timeout")
    _same(gpu, orc, 1, "after timeout (previous)")

    gpu.set_spin_limit(1 << 22)
    gpu.step(dt, 2)
    assert orc.step(dt, 2) == O.OK
    _same(gpu, orc, 0, "recovered")
    _same(gpu, orc, 1, "recovered (previous)")


def test_spin_limit_range():
    gpu = qmc.QMC(4, 1, 1, 100)
    with pytest.raises(qmc.QmcError) as ei:
        gpu.set_spin_limit((1 << 30) + 1)
    assert ei.value.code == qmc.ERR_INVALID_ARG
    gpu.set_spin_limit(1)
    gpu.set_spin_limit(1 << 22)
