"""Device memory of a context: the default stream-ordered pool and a
caller-supplied allocator (torch's caching allocator through the
qmc_config.alloc / free callbacks).

* Buffers that grow inside a qmc_step call (a capacity hint far too small)
  give the same populations as a run sized right from the start, with either
  allocator; a small-capacity run matches the oracle.
* With the callbacks, every block the library holds came from them and is
  returned to them when the context is destroyed; torch accounts for it.
* A batch context takes the allocator too.
"""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2502_18929_gb300 import problems as P
from paper_2502_18929_gb300 import qmc

pytestmark = pytest.mark.gpu


def _run(prob, rho0, nvec, seed, n_diag, dt, nsteps, **kw):
    sim = qmc.QMC(prob.n, nvec, seed, n_diag, **kw)
    sim.load_schedule(prob)
    sim.init_populations(rho0)
    sim.step(dt, nsteps)
    return sim


def _same(a, b, nvec):
    for s in range(nvec):
        for x, y in zip(a.export(s), b.export(s)):
            assert np.array_equal(x, y), s


def test_growth_in_stream_order():
    """Populations that outgrow their buffers inside one qmc_step call: 3e4
    states of one walker each spread over 10 qubits, mixed by the Hadamard
    pulse, add thousands of new states per step."""
    prob = P.ghz_circuit(10)
    rng = np.random.default_rng(3)
    states = sorted({(int(a), int(b)) for a, b in rng.integers(0, 1 << 10, size=(30000, 2))})
    rho0 = [(a, b, 1.0, 0.0) for a, b in states]
    sized = _run(prob, rho0, 4, 7, 1, 0.01, 100, capacity_hint=1 << 23)
    small = _run(prob, rho0, 4, 7, 1, 0.01, 100, capacity_hint=16)
    assert sized.counters()["redo_launches"] == 0
    assert small.counters()["redo_launches"] > 0   # buffers grew inside the step call
    _same(sized, small, 4)
    m = small.memory()
    assert m["bytes"] > 0 and m["blocks"] > 10


def test_small_capacity_matches_oracle():
    prob = P.ghz_circuit(5)
    rho0 = P.rho_basis(0)
    sim = _run(prob, rho0, 2, 3, 3000, 0.01, 80, capacity_hint=16)
    orc = O.OracleSim(prob, 2, 3, integrator=O.AB2, n_diag=3000)
    orc.init(rho0)
    assert orc.step(0.01, 80) == O.OK
    for s in range(2):
        for x, y in zip(sim.export(s), orc.population(s)):
            assert np.array_equal(x, y), s


def test_torch_allocator_callbacks():
    prob = P.ghz_circuit(5)
    rho0 = P.rho_basis(0)
    base = _run(prob, rho0, 3, 11, 5000, 0.01, 80, capacity_hint=16)
    alloc = qmc.TorchAllocator()
    torch.cuda.synchronize()
    before = torch.cuda.memory_allocated()
    sim = _run(prob, rho0, 3, 11, 5000, 0.01, 80, capacity_hint=16, allocator=alloc)
    _same(base, sim, 3)
    held = sim.memory()
    assert alloc.calls[0] > 0
    assert alloc.calls[0] - alloc.calls[1] == held["blocks"]
    assert torch.cuda.memory_allocated() - before >= held["bytes"]
    sim.close()
    torch.cuda.synchronize()
    assert alloc.calls[0] == alloc.calls[1]
    assert torch.cuda.memory_allocated() == before


def test_batch_context_takes_the_allocator():
    probs = [P.ghz_circuit(4), P.ghz_circuit(6)]
    alloc = qmc.TorchAllocator()
    a = qmc.QMC.batch(probs, [2, 3], [5, 6], [3000, 4000], capacity_hint=64)
    b = qmc.QMC.batch(probs, [2, 3], [5, 6], [3000, 4000], capacity_hint=64, allocator=alloc)
    for sim in (a, b):
        sim.init_populations(P.rho_basis(0))
        sim.step(0.01, 100)
    _same(a, b, 5)
    assert alloc.calls[0] > 0 and b.memory()["blocks"] == alloc.calls[0] - alloc.calls[1]
    b.close()
    assert alloc.calls[0] == alloc.calls[1]
