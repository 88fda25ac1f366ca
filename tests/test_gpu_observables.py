"""Per-vector observables on the GPU against the oracle (exact integers):

* N^diag <Z_q> after every step of a call (fused into the merge), and the
  sign-problem phase theta from the exact per-step N^diag;
* the batched overlap of every vector with a target state (one launch), bit
  for bit against the per-vector overlap and against the same sum over the
  oracle's populations;
* the exact anti-Hermiticity ||N - N^dagger||_F^2 of every vector.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2502_18929_gb300 import problems as P
from paper_2502_18929_gb300 import qmc

pytestmark = pytest.mark.gpu


def _pair(prob, nseg, seed, n_diag, max_ctas=0):
    gpu = qmc.QMC(prob.n, nseg, seed, n_diag, integrator=qmc.AB2, max_ctas=max_ctas)
    gpu.load_schedule(prob)
    orc = O.OracleSim(prob, nseg, seed, integrator=O.AB2, n_diag=n_diag)
    return gpu, orc


def _host_overlap(keys, re, im, n, psi):
    """The overlap's fixed-order sum over a host copy of one vector."""
    table = {int(k): (int(a), int(b)) for k, a, b in zip(keys, re, im)}
    idx = list(psi.keys())
    vals = [complex(v) for v in psi.values()]
    sr = si = 0.0
    for a in range(len(idx)):
        for b in range(len(idx)):
            nr, ni = table.get((idx[a] << n) | idx[b], (0, 0))
            nr, ni = float(nr), float(ni)
            car, cai = vals[a].real, -vals[a].imag
            pr = car * nr - cai * ni
            pi = car * ni + cai * nr
            sr += pr * vals[b].real - pi * vals[b].imag
            si += pr * vals[b].imag + pi * vals[b].real
    return complex(sr, si)


def test_z_history_and_theta_per_step():
    prob = P.ghz_circuit(4)
    gpu, orc = _pair(prob, 6, 17, 5000)
    rho0 = P.rho_pure({0: 1.0, 5: 0.4j, 9: -0.3})
    gpu.init_populations(rho0)
    orc.init(rho0)
    for call, nsteps in enumerate((40, 1, 75)):
        gpu.step(0.01, nsteps)
        zh = gpu.z_history()
        th = gpu.theta_history()
        assert zh.shape == (nsteps, 6, 4) and th.shape == (nsteps, 6)
        for k in range(nsteps):
            assert orc.step(0.01, 1) == O.OK
            for s in range(6):
                assert np.array_equal(zh[k, s], orc.zsum(s)), (call, k, s)
                _, _, dre, dim = orc.stats(s)
                assert th[k, s] == np.arctan2(float(dim), float(dre))


def test_z_history_batch_of_mixed_sizes():
    probs = [P.ghz_circuit(3), P.ghz_circuit(5), P.ghz_circuit(4)]
    seeds, nd = [3, 4, 5], [3000, 2000, 4000]
    batch = qmc.QMC.batch(probs, [2, 1, 3], seeds, nd)
    batch.init_populations(P.rho_basis(0))
    batch.step(0.01, 60)
    zh = batch.z_history()
    assert zh.shape == (60, 6, 5)
    seg = 0
    for i, pr in enumerate(probs):
        orc = O.OracleSim(pr, [2, 1, 3][i], seeds[i], integrator=O.AB2, n_diag=nd[i])
        orc.init(P.rho_basis(0))
        assert orc.step(0.01, 60) == O.OK
        for v in range(orc.nseg):
            assert np.array_equal(zh[-1, seg, :pr.n], orc.zsum(v))
            assert np.all(zh[-1, seg, pr.n:] == 0)
            seg += 1


def test_overlap_all_matches_per_vector_and_oracle():
    prob = P.ghz_circuit(4)
    gpu, orc = _pair(prob, 7, 23, 6000)
    gpu.init_populations(P.rho_basis(0))
    orc.init(P.rho_basis(0))
    gpu.step(0.01, 330)
    assert orc.step(0.01, 330) == O.OK
    for psi in (P.ghz_target(4), P.w_state(4), {0: 0.3 + 0.1j, 5: -0.2j, 15: 0.9, 6: 0.05}):
        allv = gpu.overlap_all(psi)
        for s in range(7):
            assert allv[s] == gpu.overlap(s, psi)
            assert allv[s] == _host_overlap(*orc.population(s), 4, psi)


def _spread_pairs(n, count, seed):
    """Random states plus transposed partners for a third of them (values
    differing, so the difference is nonzero), diagonal states with an
    imaginary part, sorted and merged."""
    rng = np.random.default_rng(seed)
    x = rng.integers(0, 1 << n, size=count, dtype=np.uint64)
    y = rng.integers(0, 1 << n, size=count, dtype=np.uint64)
    nn = np.uint64(n)
    keys = np.concatenate([(x << nn) | y, (y[: count // 3] << nn) | x[: count // 3], (x[:50] << nn) | x[:50]])
    keys, first = np.unique(keys, return_index=True)
    re = rng.integers(-2**31 + 1, 2**31 - 1, size=len(keys)).astype(np.int32)
    im = rng.integers(-2**31 + 1, 2**31 - 1, size=len(keys)).astype(np.int32)
    re[(re == 0) & (im == 0)] = 1
    return keys, re, im


@pytest.mark.parametrize("max_ctas", [0, 5])
def test_antihermiticity_exact(max_ctas):
    prob = P.ghz_circuit(32)
    gpu, orc = _pair(prob, 4, 1, 10**6, max_ctas=max_ctas)
    pops = [_spread_pairs(32, 3000 + 500 * s, 7 + s) for s in range(4)]
    pops[2] = (pops[2][0][:0], pops[2][1][:0], pops[2][2][:0])   # an empty vector
    gpu.set_populations(pops)
    for s, (k, r, i) in enumerate(pops):
        orc.set_population(s, k, r, i)
    got = gpu.antihermiticity()
    assert got == [orc.antiherm(s) for s in range(4)]
    assert got[2] == 0 and max(got) > 2**64


def test_antihermiticity_after_steps():
    prob = P.ghz_circuit(4)
    gpu, orc = _pair(prob, 5, 31, 4000)
    gpu.init_populations(P.rho_basis(0))
    orc.init(P.rho_basis(0))
    gpu.step(0.01, 250)
    assert orc.step(0.01, 250) == O.OK
    assert gpu.antihermiticity() == [orc.antiherm(s) for s in range(5)]


def test_antihermiticity_of_replica_sums():
    prob = P.ghz_circuit(32)
    gpu, orc = _pair(prob, 5, 2, 10**6)
    pops = [_spread_pairs(32, 2000 + 300 * s, 40 + s) for s in range(5)]
    # shared keys across vectors (some cancel in the sum), transposed keys in other vectors
    k0, r0, i0 = pops[0]
    for s in (1, 3):
        k, r, i = pops[s]
        keys = np.concatenate([k, k0[:400], ((k0[400:700] & np.uint64(0xFFFFFFFF)) << np.uint64(32)) |
                               (k0[400:700] >> np.uint64(32))])
        re = np.concatenate([r, -r0[:400], r0[400:700]])
        im = np.concatenate([i, i0[:400], i0[400:700]])
        keys, first = np.unique(keys, return_index=True)
        re, im = re[first], im[first]
        keep = (re != 0) | (im != 0)
        pops[s] = (keys[keep], re[keep], im[keep])
    gpu.set_populations(pops)
    for s, (k, r, i) in enumerate(pops):
        orc.set_population(s, k, r, i)
    for segs in ([0, 1, 2, 3, 4], [3, 0], [4], [1, 3]):
        assert gpu.antihermiticity_sum(segs) == orc.antiherm_sum(segs), segs
    with pytest.raises(qmc.QmcError):
        gpu.antihermiticity_sum([1, 1])
