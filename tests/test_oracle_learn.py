"""Pins of the FP64 training reference of the learned proposal (oracle/learn.py):

* the analytic gradient against central finite differences of the loss
  (an independent numerical derivative);
* the loss in closed form: uniform logits give log(#present outputs) per
  event, a one-hot target gives -log_softmax from scipy;
* training events against the dense Liouvillian of Eq. (2): the heat-bath
  share of every present destination equals |Re L| + |Im L| of the dense
  matrix element over its sum (quantisation and float32 rounding aside).
"""
import numpy as np
import pytest
from scipy.special import log_softmax

from oracle import dense as Dn
from oracle import learn as Lr
from oracle import oracle as O
from paper_2502_18929_gb300 import problems as P


def _tiny(seed, I=5, H=4, G=6, E=9):
    rng = np.random.default_rng(seed)
    params = {"w1": rng.standard_normal((H, I)), "b1": rng.standard_normal(H) * 0.3,
              "w2": rng.standard_normal((H, H)), "b2": rng.standard_normal(H) * 0.3,
              "w3": rng.standard_normal((G, H)), "b3": rng.standard_normal(G) * 0.3}
    feat = rng.integers(0, 2, size=(I, E)).astype(np.float64)
    feat[-1] = rng.uniform(0, 3, size=E)
    target = np.full((G, E), -1.0)
    for e in range(E):
        pres = rng.choice(G, size=int(rng.integers(1, G + 1)), replace=False)
        p = rng.uniform(0, 1, size=len(pres))
        target[pres, e] = p / p.sum()
    weight = rng.integers(1, 5, size=E).astype(np.float64)
    return params, feat, target, weight


def test_gradient_matches_finite_differences():
    params, feat, target, weight = _tiny(1)
    loss, g = Lr.loss_grad(params, feat, target, weight)
    flat = Lr.pack(params)
    gflat = Lr.pack(g)
    h = 1e-6
    num = np.zeros_like(flat)
    for i in range(flat.size):
        up, dn = flat.copy(), flat.copy()
        up[i] += h
        dn[i] -= h
        lu, _ = Lr.loss_grad(Lr.split_params(up, 5, 4, 6), feat, target, weight)
        ld, _ = Lr.loss_grad(Lr.split_params(dn, 5, 4, 6), feat, target, weight)
        num[i] = (lu - ld) / (2 * h)
    err = np.abs(num - gflat).max() / np.abs(num).max()
    assert err < 1e-6, err
    assert loss > 0


def test_uniform_logits_give_log_of_present_count():
    params, feat, target, weight = _tiny(2)
    params["w3"][:] = 0.0
    params["b3"][:] = 0.0
    loss, _ = Lr.loss_grad(params, feat, target, weight)
    npres = (target >= 0).sum(axis=0)
    ref = (weight * np.log(npres)).sum() / weight.sum()
    assert abs(loss - ref) < 1e-12


def test_one_hot_target_is_log_softmax():
    params, feat, target, weight = _tiny(3, E=6)
    G, E = target.shape
    target[:] = -1.0
    present = [np.arange(G) if e % 2 == 0 else np.arange(0, G, 2) for e in range(E)]
    for e, pres in enumerate(present):
        target[pres, e] = 0.0
        target[pres[-1], e] = 1.0
    loss, _ = Lr.loss_grad(params, feat, target, weight)
    W1, b1, W2, b2, W3, b3 = (params[k] for k in ("w1", "b1", "w2", "b2", "w3", "b3"))
    ref = 0.0
    for e, pres in enumerate(present):
        h1 = np.maximum(W1 @ feat[:, e] + b1, 0)
        h2 = np.maximum(W2 @ h1 + b2, 0)
        z = (W3 @ h2 + b3)[pres]
        ref += weight[e] * -log_softmax(z)[-1]
    assert abs(loss - ref / weight.sum()) < 1e-12


def test_sample_indices():
    assert np.array_equal(Lr.sample_indices(5, 8), np.arange(5))
    idx = Lr.sample_indices(1000, 7)
    assert np.array_equal(idx, [0, 142, 285, 428, 571, 714, 857])


@pytest.mark.parametrize("t", [1.5, 0.4])
def test_events_match_dense_heat_bath(t):
    """GHZ-3 inside the CNOT(0 -> 1) window (t = 1.5) and the Hadamard window
    (t = 0.4); one output in three removed (their targets are -1)."""
    prob = P.ghz_circuit(3)
    op = O.OracleProblem(prob)
    masks = P.destination_masks(prob)
    outs = masks[np.arange(len(masks)) % 3 != 2]
    dt = 0.01
    pops = [(np.array([0, 9, 22, 63], dtype=np.uint64), np.array([3, -1, 0, 2], np.int32),
             np.array([0, 2, -1, 0], np.int32)),
            (np.array([5, 46], dtype=np.uint64), np.array([1, 0], np.int32), np.array([0, 1], np.int32))]
    feat, target, weight = Lr.events(op, pops, t, dt, outs, 64)
    n, D = 3, 8
    Lm = Dn.liouvillian(prob, t)
    smask, sw = op.static(t, dt)
    stat = {int(m): int(w) for m, w in zip(smask, sw)}
    keys = np.concatenate([p[0] for p in pops])
    walkers = np.concatenate([np.abs(p[1]) + np.abs(p[2]) for p in pops])
    for e, key in enumerate(keys):
        x, y = int(key) >> n, int(key) & (D - 1)
        assert np.array_equal(feat[:n, e], [(x >> i) & 1 for i in range(n)])
        assert np.array_equal(feat[n:2 * n, e], [(y >> i) & 1 for i in range(n)])
        assert feat[2 * n, e] == np.float32(t)
        E = np.zeros((D, D), dtype=np.complex128)
        E[x, y] = 1.0
        M = Dn.unvec(Lm @ Dn.vec(E), D)
        share = {}
        for xx in range(D):
            for yy in range(D):
                v = M[xx, yy]
                mk = ((x ^ xx) << n) | (y ^ yy)
                share[mk] = share.get(mk, 0.0) + abs(v.real) + abs(v.imag)
        pres = [g for g, m in enumerate(outs) if stat.get(int(m), 0) > 0]
        W = sum(share.get(int(outs[g]), 0.0) for g in pres)
        for g in range(len(outs)):
            if g in pres:
                ref = share.get(int(outs[g]), 0.0) / W if W > 0 else 0.0
                assert abs(target[g, e] - ref) < 1e-6, (e, g, target[g, e], ref)
            else:
                assert target[g, e] == -1.0
        assert weight[e] == (walkers[e] if W > 0 else 0)


def test_tc_network_gradient_finite_differences():
    """The tensor-core network's reference gradient (GELU, smooth form)
    against central differences of its own loss."""
    from oracle import learn as Lr
    rng = np.random.default_rng(3)
    I, H, G, E = 9, 16, 6, 40
    params = {"w1": rng.normal(size=(H, I)) * 0.5, "b1": rng.normal(size=H) * 0.1,
              "w2": rng.normal(size=(H, H)) * 0.4, "b2": rng.normal(size=H) * 0.1,
              "w3": rng.normal(size=(G, H)) * 0.4, "b3": rng.normal(size=G) * 0.2}
    feat = np.vstack([rng.integers(0, 2, size=(I - 1, E)).astype(np.float64), rng.uniform(0, 3, size=(1, E))])
    target = rng.dirichlet(np.ones(G), size=E).T
    target[rng.random((G, E)) < 0.2] = -1.0
    weight = rng.integers(1, 5, size=E).astype(np.float64)
    loss, grad = Lr.loss_grad_tc(params, feat, target, weight, round_bf16=False)
    h = 1e-6
    for name in ("w1", "b1", "w2", "b2", "w3", "b3"):
        flat = params[name].ravel()
        for idx in rng.choice(flat.size, size=min(6, flat.size), replace=False):
            up = {k: v.copy() for k, v in params.items()}
            dn = {k: v.copy() for k, v in params.items()}
            up[name].ravel()[idx] += h
            dn[name].ravel()[idx] -= h
            num = (Lr.loss_grad_tc(up, feat, target, weight, False)[0] -
                   Lr.loss_grad_tc(dn, feat, target, weight, False)[0]) / (2 * h)
            assert abs(num - grad[name].ravel()[idx]) < 1e-6 * max(1.0, abs(num)), (name, idx)


def test_bf16_rounding():
    from oracle import learn as Lr
    # exactly representable values stay; halfway cases go to even
    vals = np.array([1.0, -2.5, 1.0 + 2**-7, 1.0 + 2**-8, 1.0 + 3 * 2**-8, 3.14159265], dtype=np.float32)
    got = Lr.bf16(vals)
    assert got[0] == 1.0 and got[1] == -2.5 and got[2] == 1.0 + 2**-7
    assert got[3] == 1.0            # halfway between 1 and 1 + 2^-7: even
    assert got[4] == 1.0 + 2**-6    # halfway between 1 + 2^-7 and 1 + 2^-6: even
    assert abs(got[5] - 3.140625) < 1e-12
