"""The benchmark's headline step at full size, checked on sampled outputs.

64 vectors of about 1.56e6 distinct random 32-qubit states (1e8 records in
N(t), about as many in N(t - dt)), one AB2 step under the GHZ-32 Liouvillian
inside the CNOT 4 -> 5 pulse, in the launch configuration bench.py times.  The
oracle cannot step 1e8 parents in a test, so it computes sampled outputs one
key at a time (the value the step leaves at a key, replayed from every parent
of N(t) and N(t - dt) that can reach it): for two vectors, about 2000 keys of
the GPU's output each and as many keys the GPU left empty must match exactly.
N(t - dt) after the step must equal the input N(t) record for record, and the
step must have taken the bucket sort (the spawn sort's path at this size).
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2502_18929_gb300 import problems as P
from paper_2502_18929_gb300 import qmc

pytestmark = pytest.mark.gpu

N_QUBITS, NSEG, PER = 32, 64, 10**8 // 64
SAMPLED = (0, 37)


def _pops(count, seed0):
    return [P.spread_population(N_QUBITS, count, seed0 + 10 * s) for s in range(NSEG)]


def _packed(pops):
    counts = np.array([len(p[0]) for p in pops], dtype=np.int64)
    return (counts, np.concatenate([p[0] for p in pops]), np.concatenate([p[1] for p in pops]),
            np.concatenate([p[2] for p in pops]))


def test_spread32_full_size_sampled_against_oracle():
    import torch
    torch.cuda.init()
    prob = P.ghz_circuit(N_QUBITS)
    seed, dt, t = 1000, 0.01, 5.3
    cur = _pops(PER, 0)
    prev = _pops(PER - 777, 5)
    gpu = qmc.QMC(N_QUBITS, NSEG, seed, PER, integrator=qmc.AB2,
                  stream=torch.cuda.current_stream().cuda_stream, capacity_hint=int(1.3 * NSEG * PER))
    gpu.load_schedule(prob)
    gpu.set_populations_packed(*_packed(cur), which=0)
    gpu.set_populations_packed(*_packed(prev), which=1)
    gpu.set_clock(530, t, t - dt, dt, True)
    gpu.counters(reset=True)
    gpu.step(dt, 1)
    c = gpu.counters()
    assert c["steps"] == 1 and c["k_cur"] == NSEG * PER and c["k_prev"] == NSEG * (PER - 777)
    assert c["sort_bucket_steps"] == 1 and c["sort_lsd_steps"] == 0
    assert c["spawns"] > 10**6

    orc = O.OracleSim(prob, NSEG, seed, integrator=O.AB2, n_diag=PER)
    for s in SAMPLED:
        orc.set_population(s, *cur[s], which=0)
        orc.set_population(s, *prev[s], which=1)
    orc.set_clock(530, t, t - dt, dt, True)
    masks, _ = O.OracleProblem(prob).static(t, 1.5 * dt)
    rng = np.random.default_rng(4)
    for s in SAMPLED:
        # N(t - dt) after the step is the input N(t)
        for a, b in zip(gpu.export(s, which=1), cur[s]):
            assert np.array_equal(a, b)
        keys, re, im = gpu.export(s)
        out = dict(zip(keys.tolist(), zip(re.tolist(), im.tolist())))
        # occupied outputs, including new states reached by spawns
        for i in rng.choice(len(keys), size=2000, replace=False):
            k = int(keys[i])
            assert orc.next_value(s, dt, k) == out[k], (s, k)
        new = np.setdiff1d(keys, cur[s][0])
        for k in rng.choice(new, size=min(300, len(new)), replace=False):
            assert orc.next_value(s, dt, int(k)) == out[int(k)], (s, int(k))
        # states the step left empty: parents that died or were annihilated,
        # and neighbours of parents that nothing reached
        gone = np.setdiff1d(cur[s][0], keys)
        probe = list(rng.choice(gone, size=min(1000, len(gone)), replace=False))
        for p in rng.choice(cur[s][0], size=1000, replace=False):
            q = int(p) ^ int(masks[rng.integers(len(masks))])
            if q not in out:
                probe.append(q)
        for k in probe:
            assert orc.next_value(s, dt, int(k)) == (0, 0), (s, int(k))
