"""Pins of the oracle's per-vector observables beyond K, N_tot and N^diag.

* <Z_q> [walker averaging, Eq. (3): rho = N / N^diag]: the oracle's integer
  sum over diagonal records of Re N_xx (-1)^(x_q) against Tr(Z_q N) with Z_q
  built as a Kronecker product (qubit q is bit q of the basis index).
* Anti-Hermiticity [End Matter on Hermiticity preservation]:
  ||N - N^dagger||_F^2 against the dense matrix norm for small n, and against
  a brute-force sum over a dictionary of entries for large values (where the
  exact sum needs more than 64 bits).
"""
import numpy as np

from oracle import oracle as O
from paper_2502_18929_gb300 import problems as P


def _zq(n, q):
    Z = np.diag([1.0, -1.0])
    I = np.eye(2)
    m = np.array([[1.0]])
    for p in range(n - 1, -1, -1):     # leftmost factor is the highest bit
        m = np.kron(m, Z if p == q else I)
    return m


def _evolved(prob, nseg, seed, nsteps, dt=0.01, n_diag=3000):
    sim = O.OracleSim(prob, nseg, seed, integrator=O.AB2, n_diag=n_diag)
    sim.init(P.rho_pure({0: 1.0, 1: 0.5j, 3: -0.3}))
    assert sim.step(dt, nsteps) == O.OK
    return sim


def test_zsum_against_kronecker_trace():
    for prob, steps in ((P.ghz_circuit(4), 150), (P.ghz_circuit(3), 230)):
        sim = _evolved(prob, 3, 5, steps)
        n = prob.n
        for s in range(3):
            N = sim.density(s)
            z = sim.zsum(s)
            for q in range(n):
                assert z[q] == int(round(np.real(np.trace(_zq(n, q) @ N)))), (s, q)


def test_antiherm_against_dense_norm():
    # complex Lindblad operators make N(t) non-Hermitian sample by sample
    from test_oracle_column import random_problem
    for prob, steps in ((P.ghz_circuit(4), 120), (random_problem(3, 4), 60)):
        sim = _evolved(prob, 3, 9, steps, dt=0.005)
        for s in range(3):
            N = sim.density(s)
            dense = np.sum(np.abs(N - N.conj().T) ** 2)
            assert sim.antiherm(s) == int(round(dense)), s


def test_antiherm_exact_beyond_64_bits():
    """Entries near 2^31 with and without transposed partners, a diagonal
    entry with an imaginary part: the exact sum exceeds 2^64."""
    n = 5
    rng = np.random.default_rng(11)
    ent = {}
    while len(ent) < 60:
        x, y = int(rng.integers(0, 32)), int(rng.integers(0, 32))
        big = 2**31 - 1 - int(rng.integers(0, 1000))
        ent[(x, y)] = (big * int(rng.choice([-1, 1])), int(rng.integers(-2**31 + 1, 2**31 - 1)))
    ent[(4, 4)] = (7, -2**31 + 1)
    keys = sorted((x << n) | y for x, y in ent)
    re = [ent[(k >> n, k & 31)][0] for k in keys]
    im = [ent[(k >> n, k & 31)][1] for k in keys]
    sim = O.OracleSim(P.pure_noise(n, 0.0, 0.0), 1, 1, n_diag=1)
    sim.set_population(0, keys, re, im)
    expect = 0
    support = set(ent) | {(y, x) for x, y in ent}
    for x, y in support:
        a = complex(*ent.get((x, y), (0, 0)))
        b = complex(*ent.get((y, x), (0, 0))).conjugate()
        d = (int(a.real) - int(b.real), int(a.imag) - int(b.imag))
        expect += d[0] * d[0] + d[1] * d[1]
    assert expect > 2**64
    assert sim.antiherm(0) == expect


def test_antiherm_sum_against_dense_norm_of_the_sum():
    """Replica aggregate: the anti-Hermiticity of the summed populations of
    several vectors (listed in any order, a vector listed once) against the
    dense norm of the summed density matrices."""
    from test_oracle_column import random_problem
    prob = random_problem(3, 6)
    sim = _evolved(prob, 5, 13, 80, dt=0.005)
    for segs in ([0, 1, 2, 3, 4], [3, 1], [2]):
        S = sum(sim.density(s) for s in segs)
        dense = np.sum(np.abs(S - S.conj().T) ** 2)
        assert sim.antiherm_sum(segs) == int(round(dense)), segs
    assert sim.antiherm_sum([4]) == sim.antiherm(4)
