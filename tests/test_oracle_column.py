"""Pin the oracle's Liouvillian columns to an independently built dense matrix.

The dense matrix is Eq. (2) assembled with Kronecker products (oracle/dense.py);
the oracle instead applies Pauli strings to the ket and bra of |x><y| term by
term.  A dropped term, a wrong sign, a missing conjugate, a transposed operand
or a wrong key packing makes some column element disagree.
"""
import math

import numpy as np
import pytest

from oracle import dense as Dn
from oracle import oracle as O
from paper_2502_18929_gb300 import problems as P


def random_problem(n, seed):
    rng = np.random.default_rng(seed)
    p = P.Problem(n=n)
    r_const = p.rate(P.RATE_CONST, 1.0)
    r_neg = p.rate(P.RATE_CONST, -0.37)          # non-Markovian (negative) rate
    r_cos = p.rate(P.RATE_COS, 0.8, 1.3, 0.2)
    letters = "IXYZ"

    def rs():
        return {q: letters[rng.integers(0, 4)] for q in range(n)}

    for _ in range(4):
        p.add_h(float(rng.normal()), rs(), int(rng.choice([r_const, r_cos])))
    for _ in range(3):
        ops = [(complex(rng.normal(), rng.normal()), rs()) for _ in range(int(rng.integers(1, 4)))]
        p.add_lindblad(ops, int(rng.choice([r_const, r_neg, r_cos])))
    return p


def oracle_dense_column(op, n, x, y, t, dte):
    D = 1 << n
    mask, qre, qim = op.column(x, y, t, dte)
    col = np.zeros(D * D, dtype=np.complex128)
    for m, a, b in zip(mask, qre, qim):
        dx, dy = int(m) >> n, int(m) & (D - 1)
        col[(x ^ dx) + D * (y ^ dy)] += (int(a) + 1j * int(b)) * 2.0**-52 / dte
    return col, mask


@pytest.mark.parametrize("n", [1, 2, 3])
@pytest.mark.parametrize("seed", range(4))
def test_columns_match_kronecker_liouvillian(n, seed):
    p = random_problem(n, seed)
    op = O.OracleProblem(p)
    t, dte = 0.3, 2.0**-7
    L = Dn.liouvillian(p, t)
    D = 1 << n
    n_terms = 2 * len(p.ham) + sum(3 * len(ops) ** 2 for ops, _, _ in p.lind)
    tol = n_terms * 2.0**-53 / dte * 2
    for x in range(D):
        for y in range(D):
            col, mask = oracle_dense_column(op, n, x, y, t, dte)
            assert np.all(np.diff(mask.astype(np.float64)) > 0), "entries not sorted by mask"
            assert np.abs(col - L[:, x + D * y]).max() < tol


def test_ghz_columns_n4():
    p = P.ghz_circuit(4)
    op = O.OracleProblem(p)
    D = 16
    for t in (0.5, 1.5, 3.5):
        L = Dn.liouvillian(p, t)
        rng = np.random.default_rng(3)
        for _ in range(40):
            x, y = int(rng.integers(0, D)), int(rng.integers(0, D))
            col, _ = oracle_dense_column(op, 4, x, y, t, 0.01)
            assert np.abs(col - L[:, x + D * y]).max() < 1e-10


def test_cnot_terms_cancel_on_control_zero():
    """The CNOT generator's X_t and Z_c X_t parts cancel when x_c = 0, so the
    column of |00><00| during the CNOT pulse has no element that flips the
    target on the ket side."""
    p = P.Problem(n=2)
    P.add_cnot_pulse(p, 0, 1, 0.0, 1.0)
    op = O.OracleProblem(p)
    mask, qre, qim = op.column(0, 0, 0.5, 0.01)
    for m, a, b in zip(mask, qre, qim):
        if int(m) == (0b10 << 2):
            assert a == 0 and b == 0
    # with the control set, the flip element is i * pi/2 * dt_eff
    mask, qre, qim = op.column(0b01, 0b01, 0.5, 0.01)
    d = {int(m): (int(a), int(b)) for m, a, b in zip(mask, qre, qim)}
    # two expanded terms (X_t and Z_c X_t), each rounded to the 2^-52 grid
    expect = 2 * round(((math.pi / 4.0) / 1.0) * (1.0 * 0.01) * 2.0**52)
    assert d[0b10 << 2] == (0, expect)
    assert d[0b10] == (0, -expect)


def test_dephasing_and_damping_elements():
    """Closed forms: dephasing gives -2 gamma_phi on coherences; amplitude
    damping moves |1><1| to |0><0| at rate gamma_1 and damps |1><1| by gamma_1."""
    g1, gp, dt = 0.03, 0.05, 0.01
    p = P.pure_noise(1, g1, gp)
    op = O.OracleProblem(p)
    mask, qre, qim = op.column(0, 1, 0.0, dt)   # rho_01
    d = {int(m): (int(a), int(b)) for m, a, b in zip(mask, qre, qim)}
    s = 2.0**52 * dt
    assert abs(d[0][0] / s - (-2 * gp - 0.5 * g1)) < 1e-12
    mask, qre, qim = op.column(1, 1, 0.0, dt)   # rho_11
    d = {int(m): (int(a), int(b)) for m, a, b in zip(mask, qre, qim)}
    assert abs(d[0][0] / s + g1) < 1e-12
    assert abs(d[(1 << 1) | 1][0] / s - g1) < 1e-12


def test_column_sum_is_trace_preserving():
    """Tr L = 0 column-wise: the diagonal destinations of any column sum to 0."""
    p = random_problem(3, 11)
    op = O.OracleProblem(p)
    for x in range(8):
        for y in range(8):
            mask, qre, qim = op.column(x, y, 0.7, 2.0**-6)
            tr = 0 + 0j
            for m, a, b in zip(mask, qre, qim):
                dx, dy = int(m) >> 3, int(m) & 7
                if (x ^ dx) == (y ^ dy):
                    tr += int(a) + 1j * int(b)
            assert abs(tr) <= 64   # a few units of 2^-52 from per-term rounding
