"""qmc_step builds the column programs of its steps while the device runs the
steps already built, copying them through pinned staging in chunks of 1, 2, 4,
... steps, with room for the call estimated from its first chunk.  A schedule
whose columns grow about tenfold partway through a call (XX, YY and ZZ terms on
every pair of qubits switch on at t = 0.155) makes the program buffer grow
inside the call (their rate a cos(omega t) makes every step's programs
distinct, so none is shared): every program is copied again and the step
graph captured again while earlier steps may still run.  The populations after the call, and
after single steps that follow it, match the oracle bit for bit."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2502_18929_gb300 import problems as P
from paper_2502_18929_gb300 import qmc


def growing_problem(n=8):
    prob = P.ghz_circuit(n)
    w = prob.window(0.155, 10.0)
    r = prob.rate(P.RATE_COS, 1.0, 2.0)   # a new column every step
    for i in range(n):
        for j in range(i + 1, n):
            for a in "XYZ":
                prob.add_h(0.02 * (1 + (i * 7 + j * 3) % 5), {i: a, j: a}, r, w)
    return prob


def test_columns_grow_inside_the_call_on_the_oracle():
    """The premise, on the CPU: the columns after t = 0.155 have many more
    destinations than before."""
    prob = growing_problem()
    op = O.OracleProblem(prob)
    before, _ = op.static(0.10, 0.015)
    after, _ = op.static(0.20, 0.015)
    assert len(after) >= 5 * len(before)


def _same(gpu, orc, nseg, where):
    for s in range(nseg):
        for which in (0, 1):
            for a, b in zip(gpu.export(s, which), orc.population(s, which)):
                assert np.array_equal(a, b), f"{where}: vector {s}, slot {which}"


@pytest.mark.gpu
def test_program_buffer_grows_inside_a_call():
    prob = growing_problem()
    nseg, seed, nd = 2, 21, 3000
    gpu = qmc.QMC(prob.n, nseg, seed, nd)
    gpu.load_schedule(prob)
    gpu.init_populations(P.rho_basis(0))
    orc = O.OracleSim(prob, nseg, seed, integrator=O.AB2, n_diag=nd)
    orc.init(P.rho_basis(0))
    m0 = gpu.memory()["bytes"]
    gpu.step(0.01, 40)
    assert orc.step(0.01, 40) == O.OK
    assert gpu.memory()["bytes"] > m0
    _same(gpu, orc, nseg, "40-step call")
    for k in range(3):
        gpu.step(0.01, 1)
        assert orc.step(0.01, 1) == O.OK
        _same(gpu, orc, nseg, f"single step {k}")
