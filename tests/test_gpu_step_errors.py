"""A step call that reaches a step whose column cannot be built (a term that
switches on at t = 0.055 with |coefficient x rate x dt_eff| >= 2^10): the steps
before it run, the call returns QMC_ERR_COEF_RANGE with the clock after them,
and both populations are those of the same steps taken without the term, bit
for bit.  The column programs of a call are built while the device runs the
earlier steps, so the failing step lies in a later chunk of the call."""
import numpy as np
import pytest

from paper_2502_18929_gb300 import problems as P
from paper_2502_18929_gb300 import qmc

pytestmark = pytest.mark.gpu


def _ctx(prob, nvec, seed, nd):
    sim = qmc.QMC(prob.n, nvec, seed, nd)
    sim.load_schedule(prob)
    sim.init_populations(P.rho_basis(0))
    return sim


def test_call_stops_before_an_unbuildable_step():
    base = P.ghz_circuit(4)
    big = P.ghz_circuit(4)
    w = big.window(0.055, 1.0)
    r = big.rate(P.RATE_CONST, 1.0)
    big.add_h(2.0 ** 17, {0: "X"}, r, w)   # 2^17 x 1.5 dt = 1966 >= 2^10 from t = 0.06 on
    a = _ctx(big, 3, 11, 2000)
    assert a.step_rc(0.01, 12) == qmc.ERR_COEF_RANGE
    step, t, t_prev, dt_last, prev_valid = a.clock()
    assert step == 6 and abs(t - 0.06) < 1e-12 and abs(t_prev - 0.05) < 1e-12 and prev_valid
    b = _ctx(base, 3, 11, 2000)
    b.step(0.01, 6)
    for s in range(3):
        for which in (0, 1):
            for x, y in zip(a.export(s, which), b.export(s, which)):
                assert np.array_equal(x, y), (s, which)
    assert a.step_history().shape[0] == 6
    # a call that fails at its first step changes nothing
    assert a.step_rc(0.01, 3) == qmc.ERR_COEF_RANGE
    assert a.clock()[0] == 6
