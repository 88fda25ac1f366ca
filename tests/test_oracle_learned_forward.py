"""Pins of the oracle's learned-proposal forward pass against mathematics it
does not share code with (the proposal is the library's extension; the paper
has none).

* ``mlp_exp`` (single-precision e^x, x <= 0) against ``numpy.exp`` within an
  error bound derived from its construction: the Lagrange remainder of the
  degree-7 Taylor polynomial of 2^f = e^{f ln 2} on [0, 1) is at most
  (ln 2)^8 / 8!, the Horner chain rounds 7 times (bounded by 16 unit
  roundoffs), and the reduced argument y = x log2(e) carries the rounding of
  the product and of the single-precision constant, each scaled by ln 2.
* The integer proposal weights Q of a source against an independent float64
  evaluation of their definition: q = softmax of the network's logits over
  the column's destinations that have an output (two ReLU layers on the bits
  of x, the bits of y and t), L_k = floor((1 - eps) q_k 2^24), S_k =
  floor(eps s_k / p_att 2^24) over the static weights s_k,
  Q_k = max(1, L_k + S_k), and the first largest Q takes the remainder so that
  sum Q = 2^24.  L_k is compared within a first-order forward error bound of
  the single-precision evaluation (each layer's accumulated rounding,
  propagated through the weights, plus the e^x bound), the rest exactly.

A transposed weight matrix, a wrong weight index, a softmax over the wrong
set, a dropped polynomial term or a wrong exponent bias each move some Q by
a relative amount far above these bounds.
"""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2502_18929_gb300 import problems as P

U = 2.0 ** -24                     # unit roundoff of single precision
C32 = float(np.float32(1.44269504))  # the single-precision log2(e) mlp_exp uses
LOG2E = 1.0 / math.log(2.0)


def exp_bound(x: float) -> float:
    """Relative error bound of mlp_exp at x <= 0 (see the module docstring)."""
    trunc = math.log(2.0) ** 8 / math.factorial(8)
    horner = 16.0 * U
    arg = math.log(2.0) * (abs(x) * abs(C32 - LOG2E) + abs(x) * LOG2E * U)
    return trunc + horner + arg


def test_mlp_exp_within_bound():
    xs = np.concatenate([-np.logspace(-8, math.log10(87.0), 4000), np.linspace(-87.0, 0.0, 20001)])
    xs = xs.astype(np.float32)
    worst = 0.0
    for x in xs:
        got = O.mlp_exp(float(x))
        ref = math.exp(float(x))
        rel = abs(got - ref) / ref
        worst = max(worst, rel / exp_bound(float(x)))
    assert worst <= 1.0, worst


def test_mlp_exp_ends():
    assert O.mlp_exp(0.0) == 1.0
    assert O.mlp_exp(-88.0) == 0.0
    # exact powers of two where f = 0: e^(-k ln 2) = 2^-k up to the argument rounding
    for k in (1, 5, 20, 60):
        x = float(np.float32(-k * math.log(2.0)))
        assert abs(O.mlp_exp(x) / math.exp(x) - 1.0) <= exp_bound(x)


def _forward_f64(net, n, x, y, t):
    """Logits of every output and first-order error bounds of the oracle's
    single-precision evaluation."""
    w1 = net["w1"].astype(np.float64)
    b1 = net["b1"].astype(np.float64)
    w2 = net["w2"].astype(np.float64)
    b2 = net["b2"].astype(np.float64)
    w3 = net["w3"].astype(np.float64)
    b3 = net["b3"].astype(np.float64)
    H = w1.shape[0]
    bits = np.array([(x >> i) & 1 for i in range(n)] + [(y >> i) & 1 for i in range(n)], dtype=np.float64)
    tf = float(np.float32(t))
    a1 = b1 + w1[:, :2 * n] @ bits + w1[:, 2 * n] * tf
    mag1 = np.abs(b1) + np.abs(w1[:, :2 * n]) @ bits + np.abs(w1[:, 2 * n] * tf)
    g1 = (2 * n + 1) * U / (1 - (2 * n + 1) * U)
    e1 = g1 * mag1
    h1 = np.maximum(a1, 0.0)
    gH = (H + 1) * U / (1 - (H + 1) * U)
    a2 = b2 + w2 @ h1
    e2 = np.abs(w2) @ e1 + gH * (np.abs(b2) + np.abs(w2) @ h1)
    h2 = np.maximum(a2, 0.0)
    z = b3 + w3 @ h2
    ez = np.abs(w3) @ e2 + gH * (np.abs(b3) + np.abs(w3) @ h2)
    return z, ez


def _check_source(sim, prob, net, x, y, t, dt_eff):
    n = prob.n
    masks, Q, p_att = sim.learned_q(x, y, t, dt_eff)
    smask, sw = O.OracleProblem(prob).static(t, dt_eff)
    assert np.array_equal(masks, smask)
    assert p_att == int(sw.sum())
    eps32 = float(np.float32(net["eps"]))
    out_index = {int(m): g for g, m in enumerate(net["out_masks"])}
    present = [k for k in range(len(masks)) if sw[k] > 0 and int(masks[k]) in out_index]
    z_all, ez_all = _forward_f64(net, n, x, y, t)
    # reference weights before the remainder
    S = np.floor(eps32 * sw.astype(np.float64) / float(p_att) * 16777216.0)
    Lref = np.zeros(len(masks))
    tol = np.zeros(len(masks))
    if present:
        z = np.array([z_all[out_index[int(masks[k])]] for k in present])
        ez = np.array([ez_all[out_index[int(masks[k])]] for k in present])
        m = z.max()
        im = int(np.argmax(z))
        e = np.exp(z - m)
        q = e / e.sum()
        eps_k = np.array([exp_bound(-(m - zk)) for zk in z]) + ez + ez[im] + U * np.abs(z - m)
        eps_q = 2.0 * eps_k.max() + (len(present) + 3) * U
        for j, k in enumerate(present):
            Lref[k] = (1.0 - eps32) * q[j] * 16777216.0
            tol[k] = Lref[k] * eps_q + 1.0
    Qpre = np.where(sw > 0, np.maximum(1.0, np.floor(Lref) + S), 0.0)
    assert int(Q.sum()) == 1 << 24
    assert np.all(Q[sw > 0] >= 1) and np.all(Q[sw == 0] == 0)
    arg = int(np.argmax(Q - np.where(sw > 0, 0, 1 << 40)))   # holder of the remainder: a largest Q
    for k in range(len(masks)):
        if sw[k] == 0 or k == arg:
            continue
        assert abs(Q[k] - Qpre[k]) <= tol[k] + 1e-9, (k, Q[k], Qpre[k], tol[k])
    # the remainder keeps the sum; it is small against the holder's weight
    rest = (1 << 24) - (Q.sum() - Q[arg])
    assert abs(rest - Qpre[arg]) <= tol[arg] + len(masks) + 2


CASES = [
    ("ghz4", lambda: P.ghz_circuit(4), [0.5, 1.5, 3.2], 0.015),
    ("ghz6", lambda: P.ghz_circuit(6), [0.2, 2.5, 5.7], 0.01),
    ("dd6", lambda: P.dd_ring(6, seed=3, t_end=4.0), [0.3, 0.51, 1.005], 0.002),
]


@pytest.mark.parametrize("name,make,times,dt", CASES)
@pytest.mark.parametrize("hidden,scale,eps", [(32, 1.0, 0.25), (64, 3.0, 0.1), (7, 2.0, 0.6)])
def test_learned_q_matches_definition(name, make, times, dt, hidden, scale, eps):
    prob = make()
    net = P.random_network(prob, hidden=hidden, seed=hidden + int(10 * scale), eps=eps, scale=scale)
    sim = O.OracleSim(prob, 1, seed=1, integrator=O.EULER, n_diag=100)
    sim.set_mlp(net)
    rng = np.random.default_rng(hidden)
    n = prob.n
    for t in times:
        for _ in range(12):
            x = int(rng.integers(0, 1 << n))
            y = int(rng.integers(0, 1 << n))
            _check_source(sim, prob, net, x, y, t, dt)


def test_learned_q_with_outputs_missing():
    """A network whose outputs cover only some destinations: the softmax runs
    over the covered ones, the others keep their static share alone."""
    prob = P.ghz_circuit(5)
    net = P.random_network(prob, hidden=16, seed=4, eps=0.3, scale=2.0)
    keep = np.arange(len(net["out_masks"])) % 3 != 1
    net = dict(net, out_masks=net["out_masks"][keep], w3=net["w3"][keep], b3=net["b3"][keep])
    sim = O.OracleSim(prob, 1, seed=1, integrator=O.EULER, n_diag=100)
    sim.set_mlp(net)
    rng = np.random.default_rng(9)
    for t in (0.5, 2.5, 4.5):
        for _ in range(10):
            _check_source(sim, prob, net, int(rng.integers(0, 32)), int(rng.integers(0, 32)), t, 0.012)
