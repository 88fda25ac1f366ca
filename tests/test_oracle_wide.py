"""Pins of the oracle at 33 <= n <= 60 qubits, where a key (x << n) | y needs
more than 64 bits.

A problem on n qubits whose terms touch only k of them is the k-qubit problem
with its qubits relabelled: its columns are the k-qubit columns with every
mask bit moved to the qubit's position, and the untouched ("spectator") bits
of x and y ride along unchanged.  If the k qubits sit at increasing positions
and the spectator bits are the same in every record, the embedding keeps the
key order, so every parent keeps its rank, draws the same random numbers, and
a whole step of the n-qubit run is the k-qubit step mapped through the
embedding.  The k-qubit oracle is pinned to the dense Kronecker Liouvillian
and the exact-mean tests, so these equalities carry those pins past 64-bit
keys: a mask shifted in 64 bits, a truncated key, or a comparison on the low
word alone breaks one of them.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2502_18929_gb300 import problems as P
from test_oracle_column import oracle_dense_column, random_problem
from oracle import dense as Dn


def embed_bits(v: int, pos) -> int:
    return sum(((v >> i) & 1) << p for i, p in enumerate(pos))


def embed_problem(small, n: int, pos):
    big = P.Problem(n=n, rates=list(small.rates), windows=list(small.windows))
    big.ham = [(h, embed_bits(xm, pos), embed_bits(zm, pos), r, w) for h, xm, zm, r, w in small.ham]
    big.lind = [([(c, embed_bits(xm, pos), embed_bits(zm, pos)) for c, xm, zm in ops], r, w)
                for ops, r, w in small.lind]
    return big


def embed_mask(m: int, k: int, n: int, pos) -> int:
    dx, dy = m >> k, m & ((1 << k) - 1)
    return (embed_bits(dx, pos) << n) | embed_bits(dy, pos)


CASES = [(33, (0, 7, 32)), (40, (1, 20, 33, 39)), (60, (5, 31, 44, 59))]


@pytest.mark.parametrize("n,pos", CASES)
def test_wide_columns_are_relabelled_small_columns(n, pos):
    k = len(pos)
    small = random_problem(k, 11 + n)
    big = embed_problem(small, n, pos)
    os_, ob = O.OracleProblem(small), O.OracleProblem(big)
    rng = np.random.default_rng(n)
    active = embed_bits((1 << k) - 1, pos)
    t, dte = 0.4, 2.0**-6
    L = Dn.liouvillian(small, t)
    D = 1 << k
    for x in range(D):
        for y in range(D):
            sx = int(rng.integers(0, 1 << 62)) & ((1 << n) - 1) & ~active
            sy = int(rng.integers(0, 1 << 62)) & ((1 << n) - 1) & ~active
            ms, re_s, im_s = os_.column(x, y, t, dte)
            mb, re_b, im_b = ob.column(embed_bits(x, pos) | sx, embed_bits(y, pos) | sy, t, dte)
            assert [embed_mask(int(m), k, n, pos) for m in ms] == [int(m) for m in mb]
            assert np.array_equal(re_s, re_b) and np.array_equal(im_s, im_b)
            # and directly against the dense Liouvillian of the active qubits
            col, _ = oracle_dense_column(os_, k, x, y, t, dte)
            assert np.abs(col - L[:, x + D * y]).max() < 1e-9
    # the static weights too
    ms, ws = os_.static(t, dte)
    mb, wb = ob.static(t, dte)
    assert sorted(embed_mask(int(m), k, n, pos) for m in ms) == [int(m) for m in mb]
    order = np.argsort([embed_mask(int(m), k, n, pos) for m in ms])
    assert np.array_equal(ws[order], wb)


def _embedded_pair(n, pos, nseg, seed, init_min, sx, sy, n_diag=3000):
    k = len(pos)
    small = P.ghz_circuit(k, gamma1=0.03, gamma_phi=0.05)
    big = embed_problem(small, n, pos)
    a = O.OracleSim(small, nseg, seed, integrator=O.AB2, init_min=init_min, n_diag=n_diag)
    b = O.OracleSim(big, nseg, seed, integrator=O.AB2, init_min=init_min, n_diag=n_diag)
    a.init(P.rho_pure({0: 1.0, 1: 0.6j, (1 << k) - 1: -0.5}))
    for s in range(nseg):
        for which in (0, 1):
            x, y, re, im = a.population_xy(s, which)
            bx = [embed_bits(int(v), pos) | sx for v in x]
            by = [embed_bits(int(v), pos) | sy for v in y]
            b.set_population_xy(s, bx, by, re, im, which)
    return a, b


def _same_embedded(a, b, nseg, pos, sx, sy):
    for s in range(nseg):
        x, y, re, im = a.population_xy(s)
        bx, by, bre, bim = b.population_xy(s)
        assert [embed_bits(int(v), pos) | sx for v in x] == [int(v) for v in bx], s
        assert [embed_bits(int(v), pos) | sy for v in y] == [int(v) for v in by], s
        assert np.array_equal(re, bre) and np.array_equal(im, bim), s


@pytest.mark.parametrize("n,pos", CASES)
@pytest.mark.parametrize("init_min", [0, 4])
def test_wide_steps_are_relabelled_small_steps(n, pos, init_min):
    k = len(pos)
    active = embed_bits((1 << k) - 1, pos)
    sx = ((0x5A5A5A5A5A5A5A5A >> 3) & ((1 << n) - 1)) & ~active
    sy = ((0x0F0F0F0F0F0F0F0F << 1) & ((1 << n) - 1)) & ~active
    nseg = 3
    a, b = _embedded_pair(n, pos, nseg, 77, init_min, sx, sy)
    for chunk in range(4):
        assert a.step(0.02, 15) == O.OK
        assert b.step(0.02, 15) == O.OK
        _same_embedded(a, b, nseg, pos, sx, sy)
    for s in range(nseg):
        st_a, st_b = a.stats(s), b.stats(s)
        assert st_a[0] == st_b[0] and st_a[1] == st_b[1]   # K and N_tot (sx != sy: no diagonal)


@pytest.mark.parametrize("n,pos", CASES[1:])
def test_wide_diagonal_observables_relabelled(n, pos):
    """With equal spectators on both sides the diagonal, <Z_q> sums and the
    anti-Hermiticity survive the embedding (spectator qubits contribute
    (-1)^(spectator bit) to Z on their own qubit)."""
    k = len(pos)
    active = embed_bits((1 << k) - 1, pos)
    sx = sy = ((0x3C3C3C3C3C3C3C3C >> 2) & ((1 << n) - 1)) & ~active
    a, b = _embedded_pair(n, pos, 2, 5, 0, sx, sy)
    assert a.step(0.02, 40) == O.OK and b.step(0.02, 40) == O.OK
    for s in range(2):
        assert np.array_equal(a.stats(s), b.stats(s))
        assert a.antiherm(s) == b.antiherm(s)
        za, zb = a.zsum(s), b.zsum(s)
        assert all(za[i] == zb[p] for i, p in enumerate(pos))
        diag = a.stats(s)[2]
        for q in range(n):
            if q not in pos:
                assert zb[q] == (-diag if (sx >> q) & 1 else diag)


def test_wide_next_value_matches_step():
    n, pos = 40, (1, 20, 33, 39)
    k = len(pos)
    active = embed_bits((1 << k) - 1, pos)
    sx, sy = (1 << 38) & ~active, (1 << 37 | 1 << 2) & ~active
    a, b = _embedded_pair(n, pos, 2, 9, 0, sx, sy)
    assert b.step(0.02, 10) == O.OK
    x, y, _, _ = b.population_xy(1)
    probes = list(zip(x[::3].tolist(), y[::3].tolist()))[:12]
    expect = [b.next_value_xy(1, 0.02, int(px), int(py)) for px, py in probes]
    assert b.step(0.02, 1) == O.OK
    x2, y2, re2, im2 = b.population_xy(1)
    got = {(int(p), int(q)): (int(r), int(i)) for p, q, r, i in zip(x2, y2, re2, im2)}
    for (px, py), e in zip(probes, expect):
        assert got.get((int(px), int(py)), (0, 0)) == e


def test_wide_init_rounding():
    """N^diag rho(0) rounded per component: every value is floor or floor + 1
    of N^diag rho, the round-up frequency matches the fractional part, and
    states whose keys differ only above bit 96 draw independently."""
    n = 60
    prob = P.Problem(n=n)
    nseg = 64
    amp = {(1 << 50): 0.5, (1 << 50) | (1 << 57): 0.5, 3: 0.5, (1 << 59) | 3: 0.5}
    rho = P.rho_pure(amp)
    sim = O.OracleSim(prob, nseg, 123, integrator=O.EULER, n_diag=1001)
    sim.init(rho)
    want = {(x, y): 1001 * complex(re, im) for x, y, re, im in rho}
    ups, tot = 0, 0
    per_key = {}
    for s in range(nseg):
        x, y, re, im = sim.population_xy(s)
        got = {(int(a), int(b)): complex(int(r), int(i)) for a, b, r, i in zip(x, y, re, im)}
        for key, v in want.items():
            g = got.get(key, 0j)
            for comp, gv in ((v.real, g.real), (v.imag, g.imag)):
                fl = np.floor(comp)
                assert gv in (fl, fl + 1), (key, comp, gv)
                if comp != fl:
                    ups += int(gv == fl + 1)
                    tot += 1
            per_key.setdefault(key, []).append(g.real - np.floor(v.real))
    # fractional parts: 1001 * 0.25 = 250.25 -> p(up) = 0.25
    assert tot > 0
    p = 0.25
    assert abs(ups / tot - p) < 3 * np.sqrt(p * (1 - p) / tot) + 1e-12
    k1, k2 = ((1 << 50), (1 << 50)), ((1 << 50) | (1 << 57), (1 << 50))
    assert per_key[k1] != per_key[k2]
