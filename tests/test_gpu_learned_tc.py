"""The learned proposal on the tensor cores (QMC_PROPOSAL_LEARNED_TC): bf16
network with fp32 accumulation and GELU.  Not reproducible bit for bit on a
CPU, so it is checked by what must hold for any proposal:

* unbiasedness: the mean density of GHZ-4 under AB2 equals the dense AB2
  recursion (every element within the family-wise bound), and one Euler step
  from a mixed state averages to (I + dt L) N over 400 vectors;
* determinism: the same seed gives the same populations, and a parent gets
  the same weights on the light and the heavy path (results do not change
  when every parent is heavy, or none);
* it really is another rule: the populations differ from the exact rule's
  and from the FP32 learned proposal's under the same seed.
"""
import numpy as np
import pytest

from oracle import dense as Dn
from paper_2502_18929_gb300 import problems as P
from paper_2502_18929_gb300 import qmc
from stat_bounds import familywise

pytestmark = pytest.mark.gpu
TC = qmc.PROPOSAL_LEARNED_TC


def _run(prob, rho0, nvec, seed, n_diag, dt, nsteps, proposal, net, integrator=qmc.AB2, heavy=256):
    gpu = qmc.QMC(prob.n, nvec, seed, n_diag, integrator=integrator)
    gpu.load_schedule(prob)
    gpu.set_mlp(net)
    gpu.set_proposal(proposal)
    gpu.set_tuning(heavy_walkers=heavy)
    gpu.init_populations(rho0)
    gpu.step(dt, nsteps)
    return gpu


def _densities(gpu, n, n_diag):
    D = 1 << n
    out = np.zeros((gpu.nseg, D, D), dtype=np.complex128)
    for s in range(gpu.nseg):
        k, r, i = gpu.export(s)
        out[s, (k >> np.uint64(n)).astype(np.int64), (k & np.uint64(D - 1)).astype(np.int64)] = r + 1j * i
    return out / n_diag


def test_tc_proposal_unbiased_ghz4():
    prob = P.ghz_circuit(4)
    net = P.random_network(prob, hidden=32, seed=3, eps=0.25, scale=2.0)
    V, nd = 64, 4000
    gpu = _run(prob, P.rho_basis(0), V, 21, nd, 0.01, 400, TC, net)
    rhos = _densities(gpu, 4, nd)
    ref = Dn.evolve(prob, Dn.rho_from_entries(4, P.rho_basis(0)), 0.01, 400, "ab2")
    se = rhos.std(0, ddof=1) / np.sqrt(V)
    sig = np.abs(ref) > 0.01
    z = np.abs(rhos.mean(0) - ref)[sig] / se[sig]
    assert z.max() < familywise(2 * sig.sum(), V), z.max()
    f = np.array([Dn.fidelity(r, P.ghz_target(4)) for r in rhos])
    assert abs(f.mean() - Dn.fidelity(ref, P.ghz_target(4))) < 3 * f.std(ddof=1) / np.sqrt(V)


def test_tc_proposal_one_step_mean():
    prob = P.ghz_circuit(3)
    rho0 = [(0, 0, 0.5, 0.0), (1, 1, 0.25, 0.0), (0, 1, 0.2, 0.1), (1, 0, 0.2, -0.1), (3, 3, 0.25, 0.0)]
    net = P.random_network(prob, hidden=16, seed=4, eps=0.05, scale=3.0)
    V, nd = 400, 4000
    gpu = qmc.QMC(3, V, 9, nd, integrator=qmc.EULER)
    gpu.load_schedule(prob)
    gpu.set_mlp(net)
    gpu.set_proposal(TC)
    gpu.init_populations(rho0)
    n0 = _densities(gpu, 3, 1)
    gpu.set_clock(250, 2.5)
    gpu.step(0.05, 1)
    n1 = _densities(gpu, 3, 1)
    Lm = Dn.liouvillian(prob, 2.5)
    pred = np.array([Dn.unvec((np.eye(64) + 0.05 * Lm) @ Dn.vec(r), 8) for r in n0])
    diff = n1 - pred
    se = diff.std(0, ddof=1) / np.sqrt(V) + 1e-9
    z = np.abs(diff.mean(0)) / se
    assert z.max() < familywise(2 * 64, V), z.max()


def test_tc_proposal_deterministic_and_path_independent():
    prob = P.ghz_circuit(5)
    net = P.random_network(prob, hidden=64, seed=8, eps=0.2, scale=1.5)
    rho0 = P.rho_pure({0: 1.0, 3: 0.5j, 17: -0.4})
    base = _run(prob, rho0, 6, 4, 30000, 0.01, 120, TC, net)
    again = _run(prob, rho0, 6, 4, 30000, 0.01, 120, TC, net)
    all_heavy = _run(prob, rho0, 6, 4, 30000, 0.01, 120, TC, net, heavy=16)
    none_heavy = _run(prob, rho0, 6, 4, 30000, 0.01, 120, TC, net, heavy=1 << 20)
    for other in (again, all_heavy, none_heavy):
        for s in range(6):
            for a, b in zip(base.export(s), other.export(s)):
                assert np.array_equal(a, b), s
    exact = _run(prob, rho0, 6, 4, 30000, 0.01, 120, qmc.PROPOSAL_EXACT, net)
    fp32 = _run(prob, rho0, 6, 4, 30000, 0.01, 120, qmc.PROPOSAL_LEARNED, net)
    for other in (exact, fp32):
        assert any(not np.array_equal(base.export(s)[0], other.export(s)[0]) or
                   not np.array_equal(base.export(s)[1], other.export(s)[1]) for s in range(6))


def test_tc_network_shape_checked():
    prob = P.ghz_circuit(4)
    gpu = qmc.QMC(4, 1, 1, 100)
    gpu.load_schedule(prob)
    gpu.set_mlp(P.random_network(prob, hidden=24, seed=1))
    with pytest.raises(qmc.QmcError):
        gpu.set_proposal(TC)
    gpu.set_proposal(qmc.PROPOSAL_LEARNED)
