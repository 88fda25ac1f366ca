"""GPU path (through the C ABI) against the CPU oracle: populations must be
bit-identical after every checked step, for every vector.

Integer work throughout (column weights in exact 2^-52 fixed point, integer
spawn counts, integer annihilation), so the bar is exact equality.
"""
import os

import numpy as np
import pytest

from oracle import oracle as O
from paper_2502_18929_gb300 import planner
from paper_2502_18929_gb300 import problems as P
from paper_2502_18929_gb300 import qmc

pytestmark = pytest.mark.gpu


def make_pair(prob, nseg, seed, n_diag, integrator=qmc.AB2, init_min=0, capacity_hint=0, max_ctas=0):
    gpu = qmc.QMC(prob.n, nseg, seed, n_diag, integrator=integrator, initiator_min=init_min,
                  capacity_hint=capacity_hint, max_ctas=max_ctas)
    gpu.load_schedule(prob)
    orc = O.OracleSim(prob, nseg, seed, integrator=integrator, init_min=init_min, n_diag=n_diag)
    return gpu, orc


def assert_same(gpu, orc, segs=None, which=0, where=""):
    for s in (range(gpu.nseg) if segs is None else segs):
        gk, gr, gi = gpu.export(s, which)
        ok, orr, oi = orc.population(s, which)
        assert gk.size == ok.size, f"{where} seg {s}: {gk.size} vs {ok.size} records"
        assert np.array_equal(gk, ok), f"{where} seg {s}: keys differ"
        assert np.array_equal(gr, orr), f"{where} seg {s}: re differs"
        assert np.array_equal(gi, oi), f"{where} seg {s}: im differs"


def test_init_bitexact():
    prob = P.ghz_circuit(4)
    rho0 = P.rho_pure({0: 1.0, 3: 0.6 - 0.3j, 9: 0.2j})
    gpu, orc = make_pair(prob, 7, 11, 997)
    gpu.init_populations(rho0)
    orc.init(rho0)
    assert_same(gpu, orc, where="init")


def test_ghz4_config_full_run():
    """GHZ-4 preparation: 16 vectors x 1e4 walkers, dt = 0.01, 400 AB2 steps,
    checked at every gate boundary and on the per-step observables."""
    prob = P.ghz_circuit(4)
    gpu, orc = make_pair(prob, 16, 2025, 10000)
    gpu.init_populations(P.rho_basis(0))
    orc.init(P.rho_basis(0))
    pl = planner.plan(prob, prob.t_end, 0.01)
    assert planner.total_steps(pl) == 400
    for piece in pl:
        planner.run(gpu, [piece])
        planner.run(orc, [piece])
        assert_same(gpu, orc, where=f"t={piece[0] + piece[1] * piece[2]:.2f}")
        hist = gpu.step_history()
        assert hist.shape[0] == piece[2]
        for s in range(16):
            assert list(hist[-1, s]) == list(orc.stats(s))
    assert gpu.clock()[0] == orc.clock()[0] == 400


def test_euler_steps():
    prob = P.ghz_circuit(3)
    gpu, orc = make_pair(prob, 5, 3, 3000, integrator=qmc.EULER)
    gpu.init_populations(P.rho_basis(0))
    orc.init(P.rho_basis(0))
    for k in range(4):
        gpu.step(0.02, 7)
        assert orc.step(0.02, 7) == O.OK
        assert_same(gpu, orc, where=f"euler chunk {k}")


def _spread_state(n, nseg, count, seed):
    pops = []
    for s in range(nseg):
        k, r, i = P.spread_population(n, count + 37 * s, seed + s)
        pops.append((k, r, i))
    return pops


def _load_state(gpu, orc, cur, prev, step, t, dt):
    gpu.set_populations(cur, which=0)
    gpu.set_populations(prev, which=1)
    gpu.set_clock(step, t, t - dt, dt, True)
    for s, (k, r, i) in enumerate(cur):
        orc.set_population(s, k, r, i, which=0)
    for s, (k, r, i) in enumerate(prev):
        orc.set_population(s, k, r, i, which=1)
    orc.set_clock(step, t, t - dt, dt, True)


def test_spread_many_tiles_ragged_n12():
    """Several sort and merge tiles per vector and a ragged tail: 3 vectors of
    ~30k random single-walker states under the DD ring, straight into AB2."""
    prob = P.dd_ring(12, seed=5, t_end=3.0)
    gpu, orc = make_pair(prob, 3, 77, 100000)
    cur = _spread_state(12, 3, 30000, 1)
    prev = _spread_state(12, 3, 29000, 50)
    _load_state(gpu, orc, cur, prev, 500, 0.2, 0.005)
    for k in range(3):
        gpu.step(0.005, 1)
        assert orc.step(0.005, 1) == O.OK
        assert_same(gpu, orc, where=f"step {k}")
        assert_same(gpu, orc, which=1, where=f"prev {k}")


def test_spread_n32_cnot_window():
    prob = P.ghz_circuit(32)
    gpu, orc = make_pair(prob, 2, 5, 10**6)
    cur = _spread_state(32, 2, 12000, 7)
    prev = _spread_state(32, 2, 11000, 70)
    _load_state(gpu, orc, cur, prev, 1234, 5.5, 0.01)
    for k in range(2):
        gpu.step(0.01, 1)
        assert orc.step(0.01, 1) == O.OK
        assert_same(gpu, orc, where=f"n32 step {k}")


def _mixed_counts_state(n, nseg, count, seed):
    """Distinct random states whose (re, im) cover every walker-pair layout of
    a light parent: one walker, both components (one or two walkers each),
    three or four walkers in one component, and a few larger parents."""
    rng = np.random.default_rng(seed)
    pops = []
    for s in range(nseg):
        k, _, _ = P.spread_population(n, count + 53 * s, seed + 100 + s)
        u = rng.random(len(k))
        sgn = lambda: rng.choice(np.array([-1, 1], np.int32), size=len(k))
        mag_small = rng.integers(1, 3, size=len(k)).astype(np.int32)
        mag_34 = rng.integers(3, 5, size=len(k)).astype(np.int32)
        mag_big = rng.integers(5, 41, size=len(k)).astype(np.int32)
        re = np.zeros(len(k), np.int32)
        im = np.zeros(len(k), np.int32)
        one = u < 0.55
        re[one & (u < 0.3)] = sgn()[one & (u < 0.3)]
        im[one & (u >= 0.3)] = sgn()[one & (u >= 0.3)]
        both = (u >= 0.55) & (u < 0.75)
        re[both] = (sgn() * mag_small)[both]
        im[both] = (sgn() * mag_small[::-1])[both]
        r34 = (u >= 0.75) & (u < 0.85)
        re[r34] = (sgn() * mag_34)[r34]
        i34 = (u >= 0.85) & (u < 0.95)
        im[i34] = (sgn() * mag_34)[i34]
        big = u >= 0.995
        re[big] = (sgn() * mag_big)[big]
        im[big & (u >= 0.998)] = (sgn() * mag_small)[big & (u >= 0.998)]
        two = (u >= 0.95) & (u < 0.995)
        re[two] = (sgn() * 2)[two]
        pops.append((k, re, im))
    return pops


def test_all_walker_pair_layouts():
    """Every layout of walker pairs in light parents (first pairs drawn per
    lane, second pairs queued, groups with larger parents on the general
    path), under AB2 with both population slots, at n = 32."""
    prob = P.ghz_circuit(32)
    gpu, orc = make_pair(prob, 3, 21, 10**6)
    cur = _mixed_counts_state(32, 3, 20000, 11)
    prev = _mixed_counts_state(32, 3, 19000, 12)
    _load_state(gpu, orc, cur, prev, 77, 5.2, 0.01)
    for k in range(3):
        gpu.step(0.01, 1)
        assert orc.step(0.01, 1) == O.OK
        assert_same(gpu, orc, where=f"pair layouts step {k}")
        assert_same(gpu, orc, which=1, where=f"pair layouts prev {k}")


@pytest.mark.parametrize("max_ctas", [1, 3, 7])
def test_many_tiles_per_cta(max_ctas):
    """Grids capped at a few CTAs: every persistent kernel runs many tiles per
    CTA (both merge staging buffers, the end marker on either stage, sort and
    merge look-back across CTAs that each hold several tiles)."""
    prob = P.ghz_circuit(32)
    gpu, orc = make_pair(prob, 2, 31, 10**6, max_ctas=max_ctas)
    cur = _spread_state(32, 2, 14000 + max_ctas, 17)
    prev = _spread_state(32, 2, 13000, 18)
    _load_state(gpu, orc, cur, prev, 999, 5.3, 0.01)
    for k in range(2):
        gpu.step(0.01, 1)
        assert orc.step(0.01, 1) == O.OK
        assert_same(gpu, orc, where=f"many tiles step {k}")


def test_spawn_sort_paths():
    """The spawn sort's two paths, each bit-exact against the oracle: random
    states (small buckets, bucket sort), and states sharing the top 16 key
    bits under a large dt, so that one bucket overflows and the step takes
    the LSD radix sort."""
    prob = P.ghz_circuit(32)
    gpu, orc = make_pair(prob, 1, 41, 10**6)
    cur = _spread_state(32, 1, 12000, 19)
    prev = _spread_state(32, 1, 11000, 20)
    _load_state(gpu, orc, cur, prev, 400, 5.1, 0.1)
    gpu.counters(reset=True)
    gpu.step(0.1, 1)
    assert orc.step(0.1, 1) == O.OK
    assert_same(gpu, orc, where="bucket sort")
    c = gpu.counters()
    assert c["sort_bucket_steps"] == 1 and c["sort_lsd_steps"] == 0

    gpu, orc = make_pair(prob, 1, 42, 10**6)
    top = np.uint64(0xBEEF) << np.uint64(48)
    low = np.uint64((1 << 48) - 1)
    packed = []
    for k, r, i in _spread_state(32, 1, 12000, 21) + _spread_state(32, 1, 11000, 22):
        k2 = np.unique((k & low) | top)
        packed.append((k2, r[:len(k2)], i[:len(k2)]))
    _load_state(gpu, orc, [packed[0]], [packed[1]], 400, 5.1, 0.1)
    gpu.counters(reset=True)
    gpu.step(0.1, 1)
    assert orc.step(0.1, 1) == O.OK
    assert_same(gpu, orc, where="LSD fallback")
    c = gpu.counters()
    assert c["sort_lsd_steps"] == 1 and c["sort_bucket_steps"] == 0


def test_spawn_sort_large_buckets():
    """States whose keys take one of 64 values in their top 12 bits: the
    step's spawns fall into a few dozen buckets of hundreds of records (the
    bucket digit is the key's top 10 to 12 bits here), each sorted by a CTA
    (buckets of more than 32 records), without overflowing into the LSD sort;
    bit-exact against the oracle."""
    prob = P.ghz_circuit(32)
    gpu, orc = make_pair(prob, 1, 43, 10**6)
    rng = np.random.default_rng(23)
    low = np.uint64((1 << 52) - 1)
    packed = []
    for k, r, i in _spread_state(32, 1, 12000, 31) + _spread_state(32, 1, 11000, 32):
        top = rng.integers(0, 64, size=k.size).astype(np.uint64) << np.uint64(52)
        k2, idx = np.unique((k & low) | top, return_index=True)
        packed.append((k2, r[idx], i[idx]))
    _load_state(gpu, orc, [packed[0]], [packed[1]], 400, 5.1, 0.1)
    gpu.counters(reset=True)
    gpu.step(0.1, 1)
    assert orc.step(0.1, 1) == O.OK
    assert_same(gpu, orc, where="large buckets")
    c = gpu.counters()
    assert c["sort_bucket_steps"] == 1 and c["sort_lsd_steps"] == 0


def test_heavy_and_light_parents():
    """A state with 1e5 walkers (four heavy chunks) next to light states."""
    prob = P.ghz_circuit(5)
    gpu, orc = make_pair(prob, 2, 9, 200000, integrator=qmc.EULER)
    keys = np.array([0, 5, (3 << 5) | 3, (31 << 5) | 31], dtype=np.uint64)
    pops = [(keys, np.array([100000, 3, -200, 1], np.int32), np.array([-7, 0, 300, -1], np.int32)),
            (keys[:2], np.array([-99999, 2], np.int32), np.array([40000, 0], np.int32))]
    gpu.set_populations(pops)
    gpu.set_clock(150, 1.5)
    for s, (k, r, i) in enumerate(pops):
        orc.set_population(s, k, r, i)
    orc.set_clock(150, 1.5)
    for k in range(3):
        gpu.step(0.01, 1)
        assert orc.step(0.01, 1) == O.OK
        assert_same(gpu, orc, where=f"heavy step {k}")


def test_initiator_mode():
    prob = P.ghz_circuit(4)
    gpu, orc = make_pair(prob, 6, 41, 10000, init_min=10)
    gpu.init_populations(P.rho_basis(0))
    orc.init(P.rho_basis(0))
    pl = planner.plan(prob, 2.5, 0.01)
    planner.run(gpu, pl)
    planner.run(orc, pl)
    assert_same(gpu, orc, where="initiator")


def test_capacity_growth_is_bit_identical():
    """Tiny initial buffers force the spawn, heavy and population buffers to grow
    and failed steps to be redone; draws are keyed by (step, vector, key,
    walker), so the result does not change."""
    prob = P.ghz_circuit(4)
    gpu, orc = make_pair(prob, 4, 8, 5000, capacity_hint=16)
    gpu.init_populations(P.rho_basis(0))
    orc.init(P.rho_basis(0))
    pl = planner.plan(prob, 2.0, 0.01)
    planner.run(gpu, pl)
    planner.run(orc, pl)
    assert_same(gpu, orc, where="growth")


def test_checkpoint_resume(tmp_path):
    prob = P.ghz_circuit(4)
    a = qmc.QMC(4, 3, 12, 4000)
    a.load_schedule(prob)
    a.init_populations(P.rho_basis(0))
    a.step(0.01, 120)
    path = str(tmp_path / "ck.bin")
    a.checkpoint(path)
    a.step(0.01, 60)
    b = qmc.QMC(4, 3, 12, 4000)
    b.load_schedule(prob)
    b.restore(path)
    b.step(0.01, 60)
    for s in range(3):
        for w in (0, 1):
            for x, y in zip(a.export(s, w), b.export(s, w)):
                assert np.array_equal(x, y)
    # a corrupted file is rejected
    raw = bytearray(open(path, "rb").read())
    raw[200] ^= 0xFF
    bad = str(tmp_path / "bad.bin")
    open(bad, "wb").write(bytes(raw))
    with pytest.raises(qmc.QmcError) as ei:
        b.restore(bad)
    assert ei.value.code == qmc.ERR_CHECKPOINT


def test_observables_and_overlap():
    prob = P.ghz_circuit(4)
    gpu, orc = make_pair(prob, 4, 31, 8000)
    gpu.init_populations(P.rho_basis(0))
    orc.init(P.rho_basis(0))
    gpu.step(0.01, 250)
    assert orc.step(0.01, 250) == O.OK
    obs = gpu.observables()
    for s in range(4):
        assert list(obs[s]) == list(orc.stats(s))
        k, r, i = orc.population(s)
        psi = P.ghz_target(4)
        expect = 0j
        for a in psi:
            for b in psi:
                key = (a << 4) | b
                j = np.searchsorted(k, key)
                if j < k.size and k[j] == key:
                    expect += complex(r[j], i[j])
        assert abs(gpu.overlap(s, psi) - expect) < 1e-9


def test_dt_too_large_is_reported_and_state_kept():
    prob = P.pure_noise(2, 0.0, 30.0)
    gpu = qmc.QMC(2, 2, 1, 500)
    gpu.load_schedule(prob)
    gpu.init_populations(P.rho_pure({0: 1.0, 3: 1.0}))
    before = [gpu.export(s) for s in range(2)]
    with pytest.raises(qmc.QmcError) as ei:
        gpu.step(0.05, 3)
    assert ei.value.code == qmc.ERR_DT_TOO_LARGE
    for s in range(2):
        for x, y in zip(before[s], gpu.export(s)):
            assert np.array_equal(x, y)
    gpu.step(0.001, 2)   # the context stays usable


def test_many_segments_two_seg_passes():
    """300 vectors: the segment id needs two radix digits."""
    prob = P.ghz_circuit(3)
    gpu, orc = make_pair(prob, 300, 4, 200)
    gpu.init_populations(P.rho_basis(0))
    orc.init(P.rho_basis(0))
    gpu.step(0.02, 30)
    assert orc.step(0.02, 30) == O.OK
    assert_same(gpu, orc, segs=[0, 1, 127, 128, 255, 256, 299], where="300 segs")


def test_dd_ring_full_size_sampled():
    """The benchmark workload at full size (12-qubit DD ring, 64 vectors x 1e6
    walkers) in the launch configuration the benchmark uses; three vectors are
    recomputed by the oracle over the first planned steps."""
    prob = P.dd_ring(12, seed=0, t_end=20.0)
    nseg, nd = 64, 10**6
    gpu, orc = make_pair(prob, nseg, 0, nd)
    gpu.init_populations(P.rho_basis(0))
    orc.init(P.rho_basis(0))
    sample = [0, 37, 63]
    orc.set_active(sample)
    pl = planner.plan(prob, prob.t_end, 0.005)
    steps = int(os.environ.get("QMC_FULLSIZE_STEPS", "24"))
    planner.run(gpu, pl, max_steps=steps)
    planner.run(orc, pl, max_steps=steps)
    assert_same(gpu, orc, segs=sample, where="dd ring full size")
    hist = gpu.step_history()
    for s in sample:
        assert list(hist[-1, s]) == list(orc.stats(s))
