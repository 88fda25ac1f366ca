"""The library's compiled column programs (term compiler + family/popcount
evaluator, the code the kernels run) against the oracle's term-by-term
columns, bit-exact, on the CPU.  Both sides take the Liouvillian of Eq. (2);
they share no code."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2502_18929_gb300 import problems as P
from paper_2502_18929_gb300 import qmc

from test_oracle_column import random_problem


def _compare(prob, x, y, t, dte):
    op = O.OracleProblem(prob)
    m_o, re_o, im_o = op.column(x, y, t, dte)
    keep = (re_o != 0) | (im_o != 0)
    m_l, re_l, im_l, P_l = qmc.column_eval(prob, x, y, t, dte)
    keep_l = (re_l != 0) | (im_l != 0)
    assert list(m_l[keep_l]) == list(m_o[keep]), (x, y)
    assert list(re_l[keep_l]) == list(re_o[keep])
    assert list(im_l[keep_l]) == list(im_o[keep])
    assert np.all(np.diff(m_l.astype(np.float64)) > 0), "library entries not in ascending mask order"
    assert P_l == int(np.abs(re_o).sum() + np.abs(im_o).sum())


@pytest.mark.parametrize("n", [1, 2, 3, 5])
@pytest.mark.parametrize("seed", range(6))
def test_random_problems(n, seed):
    prob = random_problem(n, seed)
    rng = np.random.default_rng(seed + 100)
    D = 1 << n
    for _ in range(min(64, D * D)):
        x, y = int(rng.integers(0, D)), int(rng.integers(0, D))
        _compare(prob, x, y, 0.3, 2.0**-7)


@pytest.mark.parametrize("n", [4, 12, 16, 32])
def test_ghz_circuit_all_windows(n):
    prob = P.ghz_circuit(n)
    rng = np.random.default_rng(n)
    for t in [0.5] + [k + 0.5 for k in range(1, n)]:
        for _ in range(20):
            x = int(rng.integers(0, 1 << n))
            y = int(rng.integers(0, 1 << n))
            _compare(prob, x, y, t, 0.015)


def test_dd_ring_x_basis():
    prob = P.dd_ring(12, seed=3, t_end=3.0)
    rng = np.random.default_rng(1)
    for t in (0.2, 0.505, 1.01, 1.507, 2.3):
        for _ in range(30):
            x, y = int(rng.integers(0, 4096)), int(rng.integers(0, 4096))
            _compare(prob, x, y, t, 0.0005 * 1.5)


def test_time_dependent_negative_rates():
    prob = P.ghz_circuit(6, rate_kind=P.RATE_COS, omega1=1.3, omega_phi=0.7)
    rng = np.random.default_rng(5)
    for t in (0.3, 2.4, 3.1, 4.9):   # cos(omega t) < 0 at some of these
        for _ in range(20):
            x, y = int(rng.integers(0, 64)), int(rng.integers(0, 64))
            _compare(prob, x, y, t, 0.01)


@pytest.mark.parametrize("n", [33, 40, 60])
def test_wide_programs_match_oracle(n):
    """Above 32 qubits (64-bit masks, 128-bit destination keys): the compiled
    program against the oracle's column, at random states whose bits fill all
    n qubits."""
    from test_oracle_wide import embed_problem
    rng = np.random.default_rng(n)
    pos = sorted(int(v) for v in rng.choice(n, size=4, replace=False))
    prob = embed_problem(random_problem(4, n), n, pos)
    for _ in range(24):
        x, y = int(rng.integers(0, 1 << n)), int(rng.integers(0, 1 << n))
        op = O.OracleProblem(prob)
        m_o, re_o, im_o = op.column(x, y, 0.3, 2.0**-7)
        keep = (re_o != 0) | (im_o != 0)
        m_l, re_l, im_l, P_l = qmc.column_eval(prob, x, y, 0.3, 2.0**-7)
        keep_l = (re_l != 0) | (im_l != 0)
        assert [int(v) for v in m_l[keep_l]] == [int(v) for v in m_o[keep]]
        assert list(re_l[keep_l]) == list(re_o[keep]) and list(im_l[keep_l]) == list(im_o[keep])
        assert [int(v) for v in m_l] == sorted(int(v) for v in m_l)
        assert P_l == int(np.abs(re_o).sum() + np.abs(im_o).sum())
    ghz = P.ghz_circuit(n)
    for t in (0.5, 1.5, 2.5, float(n) - 0.5):
        for _ in range(6):
            x, y = int(rng.integers(0, 1 << n)), int(rng.integers(0, 1 << n))
            _compare_wide(ghz, x, y, t, 0.01)


def _compare_wide(prob, x, y, t, dte):
    op = O.OracleProblem(prob)
    m_o, re_o, im_o = op.column(x, y, t, dte)
    keep = (re_o != 0) | (im_o != 0)
    m_l, re_l, im_l, P_l = qmc.column_eval(prob, x, y, t, dte)
    keep_l = (re_l != 0) | (im_l != 0)
    assert [int(v) for v in m_l[keep_l]] == [int(v) for v in m_o[keep]], (x, y, t)
    assert list(re_l[keep_l]) == list(re_o[keep]) and list(im_l[keep_l]) == list(im_o[keep])
    assert P_l == int(np.abs(re_o).sum() + np.abs(im_o).sum())
