"""Training of the learned proposal on the GPU (qmc_learn_*):

* training events bit-exact against the oracle's FP64 event definition
  (features, heat-bath shares of the present outputs, parent weights);
* the GPU loss and gradient (single precision, fixed-order sums) against the
  FP64 backpropagation of oracle/learn.py: relative error below 1e-5;
* Adam steps on the GPU lower the loss towards the heat-bath entropy (its
  minimum) on events logged from a plain run.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import learn as Lr  # noqa: E402
from oracle import oracle as O  # noqa: E402
from paper_2502_18929_gb300 import problems as P  # noqa: E402
from paper_2502_18929_gb300 import qmc  # noqa: E402
from paper_2502_18929_gb300 import train as T  # noqa: E402

pytestmark = pytest.mark.gpu


def _spread(n, nseg, count, seed):
    return [P.spread_population(n, count + 37 * s, seed + s) for s in range(nseg)]


def _events_pair(prob, net, pops, t, dt, max_events):
    gpu = qmc.QMC(prob.n, len(pops), 1, 1000)
    gpu.load_schedule(prob)
    gpu.set_mlp(net)
    gpu.set_populations(pops, which=0)
    gpu.set_clock(100, t)
    f, tg, w, ne = gpu.learn_events(dt, max_events)
    ref = Lr.events(O.OracleProblem(prob), pops, t, dt, net["out_masks"], max_events)
    return gpu, (f[:, :ne].cpu().numpy(), tg[:, :ne].cpu().numpy(), w[:ne].cpu().numpy(), ne), ref


@pytest.mark.parametrize("n,t,max_events", [(4, 1.5, 5000), (8, 3.3, 700), (12, 0.5, 2000)])
def test_events_match_oracle(n, t, max_events):
    prob = P.ghz_circuit(n)
    net = P.random_network(prob, hidden=8, seed=n)
    keep = np.arange(len(net["out_masks"])) % 4 != 3
    for k in ("out_masks", "w3", "b3"):
        net[k] = net[k][keep]
    pops = _spread(n, 3, 400 if n > 4 else 60, 5 + n)
    gpu, (f, tg, w, ne), (rf, rt, rw) = _events_pair(prob, net, pops, t, 0.01, max_events)
    assert ne == rf.shape[1]
    assert np.array_equal(f, rf)
    assert np.array_equal(tg, rt)
    assert np.array_equal(w, rw)


@pytest.mark.parametrize("hidden,scale", [(16, 1.0), (64, 2.0)])
def test_gradient_matches_fp64(hidden, scale):
    prob = P.ghz_circuit(6)
    net = P.random_network(prob, hidden=hidden, seed=hidden, scale=scale)
    pops = _spread(6, 2, 1500, 3)
    gpu, (f, tg, w, ne), _ = _events_pair(prob, net, pops, 2.5, 0.01, 4096)
    params = torch.tensor(T.pack(net), device="cuda")
    fd, td, wd = (torch.tensor(a, device="cuda").contiguous() for a in (f, tg, w))
    loss, grad = gpu.learn_grad(params, fd, td, wd, ne)
    G = len(net["out_masks"])
    ref_loss, ref_g = Lr.loss_grad(Lr.split_params(T.pack(net).astype(np.float64), 2 * 6 + 1, hidden, G), f, tg, w)
    gref = Lr.pack(ref_g)
    g = grad.cpu().numpy().astype(np.float64)
    assert abs(loss - ref_loss) <= 1e-6 * abs(ref_loss), (loss, ref_loss)
    rel = np.linalg.norm(g - gref) / np.linalg.norm(gref)
    assert rel < 1e-5, rel
    # every block of parameters, not just the largest
    o = 0
    for name, size in (("w1", hidden * 13), ("b1", hidden), ("w2", hidden * hidden), ("b2", hidden),
                       ("w3", G * hidden), ("b3", G)):
        blk = slice(o, o + size)
        o += size
        nb = np.linalg.norm(gref[blk])
        if nb > 0:
            assert np.linalg.norm(g[blk] - gref[blk]) / nb < 1e-4, name


def test_adam_lowers_loss_towards_entropy():
    prob = P.ghz_circuit(5)
    net = P.random_network(prob, hidden=32, seed=4, eps=0.1)
    sim = qmc.QMC(5, 8, 11, 2000)
    sim.load_schedule(prob)
    sim.set_mlp(net)
    sim.init_populations(P.rho_basis(0))
    feat, target, weight = T.collect_events(sim, 0.01, 500, 25, 2048)
    params = torch.tensor(T.pack(net), device="cuda")
    losses = T.train(sim, params, feat, target, weight, 300, lr=3e-3)
    final, _ = sim.learn_grad(params, feat, target, weight, feat.shape[1])
    # entropy of the heat-bath shares: the loss's minimum
    tg = target.cpu().numpy().astype(np.float64)
    w = weight.cpu().numpy().astype(np.float64)
    p = np.where(tg > 0, tg, 1.0)
    ent = float((w * -(np.where(tg > 0, tg * np.log(p), 0.0)).sum(axis=0)).sum() / w.sum())
    assert final < losses[0]
    assert final - ent < 0.25 * (losses[0] - ent), (losses[0], final, ent)
    # the trained parameters load into the proposal the spawn step evaluates
    sim.learn_load(params)
    sim.set_proposal(qmc.PROPOSAL_LEARNED)
    sim.step(0.01, 10)


@pytest.mark.parametrize("hidden,scale", [(16, 1.0), (64, 1.5)])
def test_tc_gradient_matches_fp64(hidden, scale):
    """The tensor-core network's loss and gradient (bf16 operands, fp32
    accumulation, GELU) against the FP64 reference with the same bf16
    roundings of weights, t and hidden activations: the remaining difference
    is the bf16 rounding of the backpropagated signals and of the weight
    products, about 1 % of the gradient's norm."""
    prob = P.ghz_circuit(6)
    net = P.random_network(prob, hidden=hidden, seed=hidden + 1, scale=scale)
    pops = _spread(6, 3, 3000, 7)
    gpu, (f, tg, w, ne), _ = _events_pair(prob, net, pops, 2.5, 0.01, 6000)
    params = torch.tensor(T.pack(net), device="cuda")
    fd, td, wd = (torch.tensor(a, device="cuda").contiguous() for a in (f, tg, w))
    loss, grad = gpu.learn_grad_tc(params, fd, td, wd, ne)
    G = len(net["out_masks"])
    ref_loss, ref_g = Lr.loss_grad_tc(Lr.split_params(T.pack(net).astype(np.float64), 13, hidden, G), f, tg, w)
    gref = Lr.pack(ref_g)
    g = grad.cpu().numpy().astype(np.float64)
    assert abs(loss - ref_loss) <= 1e-3 * abs(ref_loss), (loss, ref_loss)
    rel = np.linalg.norm(g - gref) / np.linalg.norm(gref)
    assert rel < 2e-2, rel
    o = 0
    for name, size in (("w1", hidden * 13), ("b1", hidden), ("w2", hidden * hidden), ("b2", hidden),
                       ("w3", G * hidden), ("b3", G)):
        blk = slice(o, o + size)
        o += size
        nb = np.linalg.norm(gref[blk])
        if nb > 0:
            assert np.linalg.norm(g[blk] - gref[blk]) / nb < 5e-2, name
    # deterministic: the same call gives the same bits
    loss2, grad2 = gpu.learn_grad_tc(params, fd, td, wd, ne)
    assert loss2 == loss and torch.equal(grad, grad2)


def test_tc_training_on_a_million_events():
    """Events logged over a GHZ-8 run (256 vectors, at least 10^6), full-batch Adam on the
    tensor cores: the loss falls most of the way to the heat-bath entropy,
    and the trained network runs in the tensor-core proposal."""
    prob = P.ghz_circuit(8)
    net = P.random_network(prob, hidden=64, seed=2, eps=0.1)
    sim = qmc.QMC(8, 256, 5, 200000)
    sim.load_schedule(prob)
    sim.set_mlp(net)
    sim.init_populations(P.rho_basis(0))
    sim.step(0.01, 150)
    feat, target, weight = T.collect_events(sim, 0.01, 600, 25, 1 << 20)
    E = feat.shape[1]
    assert E >= 10**6, E
    params = torch.tensor(T.pack(net), device="cuda")
    m = torch.zeros_like(params)
    v = torch.zeros_like(params)
    first = None
    for t in range(1, 151):
        loss, grad = sim.learn_grad_tc(params, feat, target, weight, E)
        first = loss if first is None else first
        sim.learn_adam(params, grad, m, v, t, 3e-3)
    final, _ = sim.learn_grad_tc(params, feat, target, weight, E)
    tg = target.cpu().numpy().astype(np.float64)
    w = weight.cpu().numpy().astype(np.float64)
    p = np.where(tg > 0, tg, 1.0)
    ent = float((w * -(np.where(tg > 0, tg * np.log(p), 0.0)).sum(axis=0)).sum() / w.sum())
    assert final - ent < 0.3 * (first - ent), (first, final, ent)
    sim.learn_load(params)
    sim.set_proposal(qmc.PROPOSAL_LEARNED_TC)
    sim.step(0.01, 10)
