"""The learned proposal's integer weights Q for given sources
(qmc_learned_weights), the handle on the network's forward pass.

* FP32 network (QMC_PROPOSAL_LEARNED): Q equals the oracle's learned_q bit
  for bit, for random sources and times (the values the step draws from).
* Tensor-core network (QMC_PROPOSAL_LEARNED_TC): Q against a float64 forward
  pass of the same bf16-rounded network (bf16 weights, inputs and hidden
  activations, GELU in its tanh form, softmax over the column's outputs):
  within 5 % of each weight plus 10^-3 of the total 2^24 (bf16 keeps 8
  significant bits; the hardware tanh is accurate to about 2^-11, so a few
  activations may round to the neighbouring bf16 value, moving a logit by
  about 10^-2), and exactly: sum Q = 2^24, Q >= 1 on every slot of positive
  width.
"""
import numpy as np
import pytest

from oracle import learn as OL
from oracle import oracle as O
from paper_2502_18929_gb300 import problems as P
from paper_2502_18929_gb300 import qmc

pytestmark = pytest.mark.gpu


def _ctx(prob, net, kind):
    gpu = qmc.QMC(prob.n, 1, 1, 1000)
    gpu.load_schedule(prob)
    gpu.set_mlp(net)
    gpu.set_proposal(kind)
    return gpu


def test_fp32_weights_match_oracle():
    prob = P.ghz_circuit(5)
    net = P.random_network(prob, hidden=32, seed=3, eps=0.25, scale=2.0)
    gpu = _ctx(prob, net, qmc.PROPOSAL_LEARNED)
    orc = O.OracleSim(prob, 1, 1, integrator=O.AB2, n_diag=1000)
    orc.set_mlp(net)
    rng = np.random.default_rng(1)
    for t, dte in ((0.3, 0.015), (1.5, 0.005), (3.7, 0.01)):
        xs = rng.integers(0, 32, size=40, dtype=np.uint64)
        ys = rng.integers(0, 32, size=40, dtype=np.uint64)
        Q = gpu.learned_weights(t, dte, xs, ys)
        for i in range(40):
            masks, q, _ = orc.learned_q(int(xs[i]), int(ys[i]), t, dte)
            want = q[q > 0]
            assert np.array_equal(Q[i][Q[i] > 0], want), (t, i)
            assert Q[i].sum() == 1 << 24


def _tc_reference(prob, net, x, y, t, dte):
    n = prob.n
    masks, w = O.OracleProblem(prob).static(t, dte)
    keep = w > 0
    masks, w = masks[keep], w[keep]
    p_att = int(w.sum())
    out_of = {int(m): g for g, m in enumerate(np.asarray(net["out_masks"], dtype=np.uint64))}
    f = np.array([(x >> q) & 1 for q in range(n)] + [(y >> q) & 1 for q in range(n)] +
                 [OL.bf16(np.float32(t))], dtype=np.float64)
    W1, W2, W3 = (OL.bf16(np.asarray(net[k], dtype=np.float32)) for k in ("w1", "w2", "w3"))
    b1, b2, b3 = (np.asarray(net[k], dtype=np.float64) for k in ("b1", "b2", "b3"))
    h1 = OL.bf16(OL.gelu(W1 @ f + b1))
    h2 = OL.bf16(OL.gelu(W2 @ h1 + b2))
    z = W3 @ h2 + b3
    g = np.array([out_of.get(int(m), -1) for m in masks])
    have = g >= 0
    eps = float(np.float32(net["eps"]))
    e = np.zeros(len(masks))
    if have.any():
        zz = z[g[have]]
        e[have] = np.exp(zz - zz.max())
    S = e.sum()
    st = np.floor(eps * w.astype(np.float64) / p_att * 2.0**24)
    L = np.floor((1.0 - eps) * e / S * 2.0**24) if S > 0 else np.zeros(len(masks))
    Q = np.maximum(1, L + st)
    Q[int(np.argmax(Q))] += 2**24 - Q.sum()
    return Q


def test_tc_weights_near_float64_forward():
    prob = P.ghz_circuit(6)
    net = P.random_network(prob, hidden=32, seed=5, eps=0.2, scale=1.5)
    gpu = _ctx(prob, net, qmc.PROPOSAL_LEARNED_TC)
    rng = np.random.default_rng(2)
    worst = 0.0
    for t, dte in ((0.4, 0.015), (2.5, 0.01)):
        xs = rng.integers(0, 64, size=48, dtype=np.uint64)
        ys = rng.integers(0, 64, size=48, dtype=np.uint64)
        Q = gpu.learned_weights(t, dte, xs, ys)
        for i in range(48):
            q = Q[i][Q[i] > 0]
            assert q.sum() == 1 << 24 and q.min() >= 1
            ref = _tc_reference(prob, net, int(xs[i]), int(ys[i]), t, dte)
            assert q.shape == ref.shape
            err = np.abs(q - ref)
            assert np.all(err <= 0.05 * ref + 2.0**24 * 1e-3), (t, i, err.max())
            worst = max(worst, float((err / 2.0**24).max()))
    print("largest |Q_gpu - Q_ref| / 2^24:", worst)
