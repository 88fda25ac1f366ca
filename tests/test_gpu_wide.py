"""The step above 32 qubits (128-bit keys) on the GPU against the oracle,
bit for bit: populations after every checked piece, N(t - dt) included, and
the observables.

* A 4-qubit GHZ circuit embedded at qubits spread over 40 and 60 (spectator
  bits set in x and y): light and heavy parents, AB2, with and without the
  initiator.
* The 40-qubit GHZ circuit from spread states: thousands of distinct keys per
  vector whose bits fill all 80 key bits, several vectors.
* Spawns crowded into few buckets: the LSD radix sort instead of the bucket
  sort, bit for bit as well.
* The counters show which paths ran; observables and target overlaps match
  the oracle's.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2502_18929_gb300 import problems as P
from paper_2502_18929_gb300 import qmc
from test_oracle_wide import embed_bits, embed_problem

pytestmark = pytest.mark.gpu


def _same(gpu, orc, nseg, which=0, where=""):
    for s in range(nseg):
        gx, gy, gr, gi = gpu.export_xy(s, which)
        ox, oy, orr, oi = orc.population_xy(s, which)
        assert gx.size == ox.size, f"{where} vector {s}: {gx.size} vs {ox.size} records"
        assert np.array_equal(gx, ox) and np.array_equal(gy, oy), f"{where} vector {s} keys"
        assert np.array_equal(gr, orr) and np.array_equal(gi, oi), f"{where} vector {s} values"


def _embedded(n, pos, sx, sy):
    k = len(pos)
    prob = embed_problem(P.ghz_circuit(k, gamma1=0.03, gamma_phi=0.05), n, pos)
    small = P.rho_pure({0: 1.0, 1: 0.6j, (1 << k) - 1: -0.5})
    rho0 = [(embed_bits(x, pos) | sx, embed_bits(y, pos) | sy, re, im) for x, y, re, im in small]
    return prob, rho0


@pytest.mark.parametrize("n,pos", [(40, (1, 20, 33, 39)), (60, (5, 31, 44, 59))])
@pytest.mark.parametrize("init_min", [0, 40])
def test_wide_embedded_ghz_parity(n, pos, init_min):
    active = embed_bits(15, pos)
    sx = ((0x5A5A5A5A5A5A5A5A >> 3) & ((1 << n) - 1)) & ~active
    sy = ((0x0F0F0F0F0F0F0F0F << 1) & ((1 << n) - 1)) & ~active
    prob, rho0 = _embedded(n, pos, sx, sy)
    nseg, nd = 5, 20000   # parents of up to 2e4 walkers: the heavy path
    gpu = qmc.QMC(n, nseg, 31, nd, integrator=qmc.AB2, initiator_min=init_min)
    gpu.load_schedule(prob)
    orc = O.OracleSim(prob, nseg, 31, integrator=O.AB2, init_min=init_min, n_diag=nd)
    gpu.init_populations(rho0)
    orc.init(rho0)
    _same(gpu, orc, nseg, where="init")
    for chunk in range(4):
        gpu.step(0.02, 25)
        assert orc.step(0.02, 25) == O.OK
        _same(gpu, orc, nseg, 0, f"chunk {chunk}")
        _same(gpu, orc, nseg, 1, f"chunk {chunk} N(t - dt)")
    obs = gpu.observables()
    for s in range(nseg):
        assert np.array_equal(obs[s], orc.stats(s)), s
    hist = gpu.step_history()
    assert hist.shape[0] == 25 and np.array_equal(hist[-1], obs)
    c = gpu.counters()
    assert c["heavy_items"] > 0 and c["steps"] == 100


def test_wide_spread_states_parity():
    """3000 distinct states whose x and y fill all 40 bits (N^diag = 1, so
    the initial values are the integers given), every vector from the same
    start with its own random stream."""
    n, nseg = 40, 4
    prob = P.ghz_circuit(n)
    rng = np.random.default_rng(7)
    xs = rng.integers(0, 1 << n, size=3000, dtype=np.uint64)
    ys = rng.integers(0, 1 << n, size=3000, dtype=np.uint64)
    states = sorted({(int(a), int(b)) for a, b in zip(xs, ys)})
    re = rng.integers(-3, 4, size=len(states))
    im = rng.integers(-2, 3, size=len(states))
    re[(re == 0) & (im == 0)] = 1
    rho0 = [(a, b, float(r), float(i)) for (a, b), r, i in zip(states, re, im)]
    gpu = qmc.QMC(n, nseg, 5, 1, integrator=qmc.AB2)
    gpu.load_schedule(prob)
    orc = O.OracleSim(prob, nseg, 5, integrator=O.AB2, n_diag=1)
    gpu.init_populations(rho0)
    orc.init(rho0)
    _same(gpu, orc, nseg, where="init")
    gpu.set_clock(500, 5.0)
    orc.set_clock(500, 5.0)
    for chunk in range(3):
        gpu.step(0.01, 2)
        assert orc.step(0.01, 2) == O.OK
        _same(gpu, orc, nseg, 0, f"chunk {chunk}")
        _same(gpu, orc, nseg, 1, f"chunk {chunk} N(t - dt)")
    c = gpu.counters()
    assert c["sort_bucket_steps"] == 6 and c["sort_lsd_steps"] == 0   # keys spread over all buckets


def test_wide_lsd_fallback_parity():
    """Spawns crowded into one bucket per vector (states that differ only in
    the low 16 bits of x and y, 40 walkers each, inside the CNOT 4 -> 5
    pulse): more than a sort window's worth of records share a bucket, so the
    step takes the LSD radix sort; bit for bit with the oracle."""
    n, nseg = 40, 2
    prob = P.ghz_circuit(n)
    rng = np.random.default_rng(11)
    xs = rng.integers(0, 1 << 16, size=2500)
    ys = rng.integers(0, 1 << 16, size=2500)
    states = sorted({(int(a), int(b)) for a, b in zip(xs, ys)})
    sign = rng.choice([-1, 1], size=len(states))
    rho0 = [(a, b, float(40 * s), float(-20 * s)) for (a, b), s in zip(states, sign)]
    gpu = qmc.QMC(n, nseg, 9, 1, integrator=qmc.AB2)
    gpu.load_schedule(prob)
    orc = O.OracleSim(prob, nseg, 9, integrator=O.AB2, n_diag=1)
    gpu.init_populations(rho0)
    orc.init(rho0)
    gpu.set_clock(500, 5.0)
    orc.set_clock(500, 5.0)
    for chunk in range(3):
        gpu.step(0.01, 2)
        assert orc.step(0.01, 2) == O.OK
        _same(gpu, orc, nseg, 0, f"chunk {chunk}")
        _same(gpu, orc, nseg, 1, f"chunk {chunk} N(t - dt)")
    c = gpu.counters()
    assert c["sort_lsd_steps"] > 0 and c["spawns"] > 6 * 2 * 1824
    obs = gpu.observables()
    for s in range(nseg):
        assert np.array_equal(obs[s], orc.stats(s)), s


def test_wide_overlap_and_rejections():
    n, pos = 40, (1, 20, 33, 39)
    prob, rho0 = _embedded(n, pos, 0, 0)
    gpu = qmc.QMC(n, 3, 2, 5000)
    gpu.load_schedule(prob)
    gpu.init_populations(rho0)
    gpu.step(0.02, 60)
    target = {embed_bits(0, pos): 2 ** -0.5, embed_bits(15, pos): 2 ** -0.5}
    ov = gpu.overlap_all(target)
    for s in range(3):
        x, y, re, im = gpu.export_xy(s)
        vals = {(int(a), int(b)): complex(int(r), int(i)) for a, b, r, i in zip(x, y, re, im)}
        want = sum(np.conj(pa) * vals.get((a, b), 0) * pb for a, pa in target.items() for b, pb in target.items())
        assert abs(ov[s] - want) < 1e-9 * max(1.0, abs(want)), s
    with pytest.raises(qmc.QmcError):
        gpu.export(0)
    with pytest.raises(qmc.QmcError):
        gpu.set_proposal(qmc.PROPOSAL_STATIC)
    with pytest.raises(qmc.QmcError):
        gpu.antihermiticity()


def test_spread40_full_size_sampled_against_oracle():
    """The 40-qubit benchmark step at full size (64 vectors of about 1.56e6
    distinct random states, 1e8 records, 128-bit keys), one AB2 step inside the
    CNOT 4 -> 5 pulse, checked on sampled outputs that the oracle computes one
    state at a time from every parent that can reach it: occupied outputs, new
    states, and states the step left empty; N(t - dt) after the step is the
    input N(t)."""
    import torch
    torch.cuda.init()
    n, nseg, per = 40, 64, 10**8 // 64
    prob = P.ghz_circuit(n)
    seed, dt, t = 1000, 0.01, 5.3
    cur = [P.spread_population_xy(n, per, 10 * s) for s in range(nseg)]
    prev = [P.spread_population_xy(n, per - 777, 5 + 10 * s) for s in range(nseg)]

    def packed(pops):
        return ([len(p[0]) for p in pops], *[np.concatenate([p[k] for p in pops]) for k in range(4)])

    gpu = qmc.QMC(n, nseg, seed, per, integrator=qmc.AB2, stream=torch.cuda.current_stream().cuda_stream,
                  capacity_hint=int(1.3 * nseg * per))
    gpu.load_schedule(prob)
    gpu.set_populations_xy(*packed(cur), which=0)
    gpu.set_populations_xy(*packed(prev), which=1)
    gpu.set_clock(530, t, t - dt, dt, True)
    gpu.counters(reset=True)
    gpu.step(dt, 1)
    c = gpu.counters()
    assert c["steps"] == 1 and c["k_cur"] == nseg * per and c["k_prev"] == nseg * (per - 777)
    assert c["spawns"] > 10**6 and c["redo_launches"] == 0

    orc = O.OracleSim(prob, nseg, seed, integrator=O.AB2, n_diag=per)
    sampled = (0, 41)
    for s in sampled:
        orc.set_population_xy(s, *cur[s], which=0)
        orc.set_population_xy(s, *prev[s], which=1)
    orc.set_clock(530, t, t - dt, dt, True)
    masks, _ = O.OracleProblem(prob).static(t, 1.5 * dt)
    rng = np.random.default_rng(4)
    ymask = (1 << n) - 1
    for s in sampled:
        px, py, pre_, pim = gpu.export_xy(s, which=1)
        assert np.array_equal(px, cur[s][0]) and np.array_equal(py, cur[s][1])
        assert np.array_equal(pre_, cur[s][2]) and np.array_equal(pim, cur[s][3])
        x, y, re, im = gpu.export_xy(s)
        out = {(int(a), int(b)): (int(r), int(i)) for a, b, r, i in zip(x, y, re, im)}
        before = set(zip(cur[s][0].tolist(), cur[s][1].tolist()))
        keys = list(out.keys())
        for i in rng.choice(len(keys), size=1500, replace=False):
            k = keys[i]
            assert orc.next_value_xy(s, dt, k[0], k[1]) == out[k], (s, k)
        new = [k for k in keys if k not in before]
        for i in rng.choice(len(new), size=min(300, len(new)), replace=False):
            k = new[i]
            assert orc.next_value_xy(s, dt, k[0], k[1]) == out[k], (s, k)
        gone = [k for k in before if k not in out]
        probe = [gone[i] for i in rng.choice(len(gone), size=min(600, len(gone)), replace=False)]
        for i in rng.choice(per, size=600, replace=False):
            m = int(masks[rng.integers(len(masks))])
            q = (int(cur[s][0][i]) ^ (m >> n), int(cur[s][1][i]) ^ (m & ymask))
            if q not in out:
                probe.append(q)
        for k in probe:
            assert orc.next_value_xy(s, dt, k[0], k[1]) == (0, 0), (s, k)
