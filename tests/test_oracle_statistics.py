"""Statistical pins of the oracle against what the paper and the mathematics fix.

* Exact mean: every spawn is unbiased [End Matter, spawn step] and annihilation is
  exact integer addition, so E[N_k] / N^diag equals the deterministic Euler / AB2
  recursion [End Matter, simulation methodology] on the same time grid.
* Closed forms: pure dephasing and amplitude damping (scalar recurrences).
* Brute force: the exact one-step law of B(m, p) x multinomial with the paper's
  sign rule, enumerated for three walkers, against the oracle's frequencies.
* Invariants: E[N^diag] constant (trace preservation), Hermiticity in mean.
* Error bound Eq. (5); initiator rule [End Matter, simulation methodology].
"""
import itertools
import math

import numpy as np
import pytest

from oracle import dense as Dn
from oracle import oracle as O
from paper_2502_18929_gb300 import problems as P
from stat_bounds import SINGLE, familywise


def run_densities(prob, rho0, V, seed, dt, nsteps, integrator=O.AB2, n_diag=10000):
    sim = O.OracleSim(prob, V, seed=seed, integrator=integrator, n_diag=n_diag)
    sim.init(rho0)
    assert sim.step(dt, nsteps) == O.OK
    return sim, np.array([sim.density(s) / n_diag for s in range(V)])


@pytest.fixture(scope="module")
def ghz4_run():
    prob = P.ghz_circuit(4)
    rho0 = P.rho_basis(0)
    sim, rhos = run_densities(prob, rho0, 16, 1, 0.01, 400)
    ref = Dn.evolve(prob, Dn.rho_from_entries(4, rho0), 0.01, 400, "ab2")
    return prob, sim, rhos, ref


def test_exact_mean_ghz4_ab2(ghz4_run):
    """GHZ-4 preparation (Fig. 1(d)), 16 vectors x 1e4 walkers, 400 AB2 steps."""
    _, _, rhos, ref = ghz4_run
    mean = rhos.mean(0)
    se = rhos.std(0, ddof=1) / np.sqrt(rhos.shape[0])
    sig = np.abs(ref) > 0.01
    z = np.abs(mean - ref)[sig] / se[sig]
    assert z.max() < familywise(2 * sig.sum(), 16), z.max()
    # fidelity to GHZ is linear in rho before the modulus: within 3 sigma
    f = np.array([Dn.fidelity(r, P.ghz_target(4)) for r in rhos])
    f_ref = Dn.fidelity(ref, P.ghz_target(4))
    assert abs(f.mean() - f_ref) < SINGLE * f.std(ddof=1) / 4
    # <Z_q> of every qubit (diagonal observables), family of 4
    D = 16
    for q in range(4):
        zq = np.array([(-1.0) ** ((np.arange(D) >> q) & 1) for _ in range(1)])[0]
        vals = np.array([np.real(np.diag(r)) @ zq for r in rhos])
        exact = np.real(np.diag(ref)) @ zq
        assert abs(vals.mean() - exact) < familywise(4, 16) * vals.std(ddof=1) / 4


def test_trace_and_hermiticity_in_mean(ghz4_run):
    _, sim, rhos, _ = ghz4_run
    tr = np.array([np.trace(r) for r in rhos])
    assert abs(tr.real.mean() - 1.0) < SINGLE * tr.real.std(ddof=1) / 4 + 1e-3
    anti = rhos - np.conj(np.transpose(rhos, (0, 2, 1)))
    se = anti.std(0, ddof=1) / 4 + 1e-12
    # real and imaginary parts of the 256 elements
    assert (np.abs(anti.mean(0).real) / se).max() < familywise(512, 16)
    assert (np.abs(anti.mean(0).imag) / se).max() < familywise(512, 16)
    # sign-problem phase stays small (the paper reports theta < 0.02 at n = 10)
    for s in range(16):
        k, ntot, dre, dim = sim.stats(s)
        assert abs(math.atan2(dim, dre)) < 0.1


def test_exact_mean_euler():
    prob = P.ghz_circuit(3)
    rho0 = P.rho_basis(0)
    _, rhos = run_densities(prob, rho0, 24, 5, 0.01, 150, integrator=O.EULER)
    ref = Dn.evolve(prob, Dn.rho_from_entries(3, rho0), 0.01, 150, "euler")
    se = rhos.std(0, ddof=1) / np.sqrt(24)
    sig = np.abs(ref) > 0.01
    assert (np.abs(rhos.mean(0) - ref)[sig] / se[sig]).max() < familywise(2 * sig.sum(), 24)


@pytest.mark.parametrize("integrator", [O.EULER, O.AB2])
def test_pure_dephasing_closed_form(integrator):
    """rho_01 obeys a' = lam a with lam = -2 gamma_phi.  Euler: a_k = (1 + lam dt)^k a_0.
    AB2 after one Euler step: a_{k+1} = a_k + dt lam (3/2 a_k - 1/2 a_{k-1}), whose
    solution is A r1^k + B r2^k with r the roots of r^2 - (1 + 3/2 h) r + h/2 = 0."""
    gp, dt, K, V, nd = 0.5, 0.01, 100, 64, 2000
    prob = P.pure_noise(1, 0.0, gp)
    rho0 = P.rho_pure({0: 1.0, 1: 1.0})
    _, rhos = run_densities(prob, rho0, V, 3, dt, K, integrator=integrator, n_diag=nd)
    lam = -2 * gp
    h = lam * dt
    if integrator == O.EULER:
        expect = 0.5 * (1 + h) ** K
    else:
        disc = math.sqrt((1 + 1.5 * h) ** 2 - 2 * h)
        r1, r2 = ((1 + 1.5 * h) + disc) / 2, ((1 + 1.5 * h) - disc) / 2
        a0, a1 = 0.5, 0.5 * (1 + h)
        B = (a1 - r1 * a0) / (r2 - r1)
        A = a0 - B
        expect = A * r1**K + B * r2**K
    vals = rhos[:, 0, 1]
    assert np.all(np.abs(vals.imag) == 0)
    se = vals.real.std(ddof=1) / np.sqrt(V)
    assert abs(vals.real.mean() - expect) < SINGLE * se
    # diagonal untouched by dephasing
    assert np.all(rhos[:, 0, 0] == 0.5) and np.all(rhos[:, 1, 1] == 0.5)


def test_amplitude_damping_closed_form():
    """rho_11 decays as (1 - gamma_1 dt)^k under Euler (single qubit T1)."""
    g1, dt, K, V, nd = 0.5, 0.01, 100, 48, 3000
    prob = P.pure_noise(1, g1, 0.0)
    _, rhos = run_densities(prob, P.rho_basis(1), V, 9, dt, K, integrator=O.EULER, n_diag=nd)
    expect = (1 - g1 * dt) ** K
    v11 = rhos[:, 1, 1].real
    assert abs(v11.mean() - expect) < SINGLE * v11.std(ddof=1) / np.sqrt(V)
    v00 = rhos[:, 0, 0].real
    assert abs(v00.mean() - (1 - expect)) < SINGLE * v00.std(ddof=1) / np.sqrt(V)


def _exact_one_step_law(prob, key_x, key_y, re, im, dt):
    """Enumerate N(t+dt) for the walkers of one parent, from the dense Eq. (2)
    column and the paper's B(m, p) x multinomial with its sign rule."""
    n = prob.n
    D = 1 << n
    L = Dn.liouvillian(prob, 0.0)
    col = L[:, key_x + D * key_y]
    # walker types: real walkers with sign sgn(re), imaginary with i sgn(im)
    events = []
    for idx in np.nonzero(np.abs(col) > 0)[0]:
        xd, yd = int(idx) % D, int(idx) // D
        dest = (xd << n) | yd
        c = col[idx]
        if c.real != 0:
            events.append((dt * abs(c.real), dest, "re", np.sign(c.real)))
        if c.imag != 0:
            events.append((dt * abs(c.imag), dest, "im", np.sign(c.imag)))
    p_spawn = sum(e[0] for e in events)
    assert p_spawn < 1
    walkers = [("re", np.sign(re))] * abs(re) + [("im", np.sign(im))] * abs(im)

    def contributions(w):
        comp, sg = w
        s = sg if comp == "re" else 1j * sg       # walker sign s in {+-1, +-i}
        out = [(1 - p_spawn, None, 0j)]
        for pe, dest, chan, sl in events:
            v = s * sl if chan == "re" else 1j * s * sl
            out.append((pe, dest, v))
        return out

    base = {(key_x << n) | key_y: complex(re, im)}
    law = {}
    for combo in itertools.product(*[contributions(w) for w in walkers]):
        pr = 1.0
        pop = dict(base)
        for pe, dest, v in combo:
            pr *= pe
            if dest is not None:
                pop[dest] = pop.get(dest, 0) + v
        state = tuple(sorted((k, int(round(v.real)), int(round(v.imag)))
                             for k, v in pop.items() if v != 0))
        law[state] = law.get(state, 0.0) + pr
    return law


def test_brute_force_one_step_distribution():
    """Chi-square of the oracle's one-step outcomes (20000 independent vectors)
    against the exactly enumerated law for 2 real + 1 imaginary walkers."""
    prob = P.Problem(n=1)
    one = prob.rate(P.RATE_CONST, 1.0)
    prob.add_h(3.0, {0: "X"}, one)
    prob.add_h(-2.0, {0: "Y"}, one)
    prob.add_h(1.5, {0: "Z"}, one)
    P.add_local_noise(prob, 2.0, 1.0)
    dt = 0.02
    kx, ky, re, im = 0, 1, 2, -1
    law = _exact_one_step_law(prob, kx, ky, re, im, dt)
    V = 20000
    sim = O.OracleSim(prob, V, seed=2024, integrator=O.EULER, n_diag=1000)
    key = (kx << 1) | ky
    for s in range(V):
        sim.set_population(s, [key], [re], [im])
    sim.set_clock(0, 0.0)
    assert sim.step(dt, 1) == O.OK
    counts = {}
    for s in range(V):
        k, r, i = sim.population(s)
        st = tuple(sorted(zip(k.tolist(), r.tolist(), i.tolist())))
        counts[st] = counts.get(st, 0) + 1
    assert set(counts) <= set(law), set(counts) - set(law)
    # chi-square over cells with expected >= 5 (the rest pooled)
    chi2, dof, pooled_e, pooled_o = 0.0, -1, 0.0, 0
    for st, pr in law.items():
        e = pr * V
        o = counts.get(st, 0)
        if e >= 5:
            chi2 += (o - e) ** 2 / e
            dof += 1
        else:
            pooled_e += e
            pooled_o += o
    if pooled_e >= 5:
        chi2 += (pooled_o - pooled_e) ** 2 / pooled_e
        dof += 1
    from scipy.stats import chi2 as chi2dist
    assert dof >= 10
    assert chi2dist.sf(chi2, dof) > 1e-4, (chi2, dof)


def test_error_bound_eq5():
    """One-step squared error (normalised by N^diag) is below Lambda 2 N_tot / (N^diag)^2."""
    prob = P.ghz_circuit(3)
    nd = 1000
    V = 400
    rng = np.random.default_rng(4)
    keys = np.unique(rng.integers(0, 64, size=12).astype(np.uint64))
    re = rng.integers(-30, 31, size=keys.size).astype(np.int32)
    im = rng.integers(-30, 31, size=keys.size).astype(np.int32)
    sim = O.OracleSim(prob, V, seed=77, integrator=O.EULER, n_diag=nd)
    for s in range(V):
        sim.set_population(s, keys, re, im)
    t, dt = 1.5, 0.01
    sim.set_clock(150, t)
    assert sim.step(dt, 1) == O.OK
    D = 8
    N0 = np.zeros((D, D), dtype=complex)
    for k, a, b in zip(keys, re, im):
        N0[int(k) >> 3, int(k) & 7] = a + 1j * b
    L = Dn.liouvillian(prob, t)
    mean_next = Dn.unvec(Dn.vec(N0) + dt * (L @ Dn.vec(N0)), D)
    err2 = np.mean([np.sum(np.abs(sim.density(s) - mean_next) ** 2) for s in range(V)]) / nd**2
    ntot = np.sum(np.abs(re)) + np.sum(np.abs(im))
    lam = 0.0
    for k in keys:
        c = L[:, (int(k) >> 3) + D * (int(k) & 7)]
        lam = max(lam, dt**2 * np.count_nonzero(np.abs(c) > 1e-15) * np.sum(np.abs(c) ** 2))
    bound = (lam + 0.25) * 2 * ntot / nd**2
    assert err2 <= bound
    assert err2 > 0


def test_initiator_rule():
    """A parent below the threshold (xi N^diag walkers) may not create new
    states; spawns onto occupied states and from initiators are kept."""
    prob = P.ghz_circuit(3)
    heavy, light = 0, (0b011 << 3) | 0b101
    V = 64

    def run(init_min):
        sim = O.OracleSim(prob, V, seed=8, integrator=O.EULER, init_min=init_min, n_diag=1000)
        for s in range(V):
            sim.set_population(s, [heavy, light], [500, 3], [0, -2])
        sim.set_clock(120, 1.2)
        assert sim.step(0.02, 1) == O.OK
        return [set(sim.population(s)[0].tolist()) for s in range(V)]

    op = O.OracleProblem(prob)
    heavy_dest = {heavy ^ int(m) for m in op.column(0, 0, 1.2, 0.02)[0]}
    light_dest = {light ^ int(m) for m in op.column(0b011, 0b101, 1.2, 0.02)[0]}
    with_rule = run(init_min=10)
    for keys in with_rule:
        assert keys <= heavy_dest | {heavy, light}
    without = run(init_min=0)
    new_from_light = set().union(*without) & (light_dest - heavy_dest - {heavy, light})
    assert new_from_light, "the light parent should create new states without the rule"


def test_split_calls_are_bit_identical():
    prob = P.ghz_circuit(3)
    a = O.OracleSim(prob, 3, seed=5, n_diag=3000)
    b = O.OracleSim(prob, 3, seed=5, n_diag=3000)
    a.init(P.rho_basis(0))
    b.init(P.rho_basis(0))
    assert a.step(0.01, 60) == O.OK
    for _ in range(3):
        assert b.step(0.01, 20) == O.OK
    for s in range(3):
        for x, y in zip(a.population(s), b.population(s)):
            assert np.array_equal(x, y)
        for x, y in zip(a.population(s, 1), b.population(s, 1)):
            assert np.array_equal(x, y)


def test_initial_rounding_unbiased():
    """N(0) = N^diag rho(0) with stochastic rounding: exact in the mean."""
    amps = {0: 1.0, 3: 0.7 + 0.2j, 5: -0.4j}
    rho0 = P.rho_pure(amps)
    V, nd = 2000, 37
    sim = O.OracleSim(P.pure_noise(3, 0.0, 0.0), V, seed=3, n_diag=nd)
    sim.init(rho0)
    target = Dn.rho_from_entries(3, rho0) * nd
    acc = np.array([sim.density(s) for s in range(V)])
    se = acc.std(0, ddof=1) / np.sqrt(V) + 1e-9
    assert (np.abs(acc.mean(0) - target) / se).max() < familywise(2 * 64, V)
    # every value is floor or ceil of the target
    fl = np.floor(target.real)
    assert np.all((acc.real == fl) | (acc.real == fl + 1))


def test_rejects_too_large_step():
    prob = P.pure_noise(1, 0.0, 30.0)
    sim = O.OracleSim(prob, 1, seed=0, n_diag=100)
    sim.init(P.rho_pure({0: 1.0, 1: 1.0}))
    assert sim.step(0.02, 1) == O.ERR_DT_TOO_LARGE


@pytest.mark.parametrize("integrator,proposal", [(O.AB2, 0), (O.EULER, 0), (O.AB2, 1)])
def test_next_value_equals_the_step(integrator, proposal):
    """The one-key form of the step (the value N(t + dt) takes at a key,
    replayed from the parents that can reach it) equals the step itself at
    every output key and at unoccupied neighbours, with the initiator rule
    on; it is what the full-size GPU check samples."""
    prob = P.ghz_circuit(5)
    sim = O.OracleSim(prob, 3, seed=19, integrator=integrator, init_min=40, n_diag=3000)
    sim.set_proposal(proposal)
    sim.init(P.rho_pure({0: 1.0, 7: 0.5, 18: -0.4j}))
    assert sim.step(0.01, 230) == O.OK
    # every state a parent of N(t) or N(t - dt) can reach: parent key ^ destination mask
    _, t, _, _, _ = sim.clock()
    masks, _ = O.OracleProblem(prob).static(t, 0.01)
    before = {}
    for s in range(3):
        parents = set(int(v) for v in sim.population(s)[0]) | set(int(v) for v in sim.population(s, 1)[0])
        probe = parents | {p ^ int(m) for p in parents for m in masks}
        before[s] = {key: sim.next_value(s, 0.01, key) for key in sorted(probe)}
    assert sim.step(0.01, 1) == O.OK
    for s in range(3):
        k, r, i = sim.population(s)
        after = {int(a): (int(b), int(c)) for a, b, c in zip(k, r, i)}
        assert set(after) <= set(before[s])
        for key, v in before[s].items():
            assert v == after.get(key, (0, 0)), (s, key)


def test_operator_form_dense_recursion_matches_kronecker():
    """The matrix-free dense recursion (operators applied to rho) equals the
    Kronecker-matrix recursion of Eq. (2), through pulse-window changes."""
    for prob, rho0, steps in ((P.ghz_circuit(3), P.rho_basis(0), 300),
                              (P.dd_ring(4, seed=2, t_end=2.0, x_basis=False), P.rho_pure(P.w_state(4)), 250)):
        r0 = Dn.rho_from_entries(prob.n, rho0)
        a = Dn.evolve(prob, r0, 0.008, steps, "ab2")
        b = Dn.evolve_operators(prob, r0, 0.008, steps, "ab2")
        assert np.abs(a - b).max() < 1e-12
