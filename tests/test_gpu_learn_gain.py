"""What the trained network gains, reported honestly.

GHZ-5 preparation under local noise, 64 vectors x N^diag = 2000, 500 steps
of dt = 0.01: the standard deviation over vectors of the final GHZ fidelity
with the plain method (exact |L|-weighted choice), the static proposal, and
the learned proposal before and after training on events logged from a plain
run.  Training must bring the loss to the heat-bath entropy and the learned
proposal's spread back to the plain method's (the untrained network's walker
counts above one inflate it); the plain method's per-walker variance is
already minimal, so no variance gain over it is expected or claimed.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2502_18929_gb300 import problems as P  # noqa: E402
from paper_2502_18929_gb300 import qmc  # noqa: E402
from paper_2502_18929_gb300 import train as T  # noqa: E402

pytestmark = pytest.mark.gpu

N, V, ND, DT, STEPS = 5, 64, 2000, 0.01, 500


def _final_fidelity(prob, net, mode, params=None):
    sim = qmc.QMC(N, V, 7, ND)
    sim.load_schedule(prob)
    if mode == qmc.PROPOSAL_LEARNED:
        sim.set_mlp(net)
        if params is not None:
            sim.learn_load(params)
    sim.set_proposal(mode)
    sim.init_populations(P.rho_basis(0))
    sim.step(DT, STEPS)
    obs = sim.observables()
    tgt = P.ghz_target(N)
    return np.array([sim.overlap(v, tgt).real / (2.0 * obs[v, 2]) for v in range(V)])


def test_trained_proposal_recovers_plain_variance():
    prob = P.ghz_circuit(N)
    net = P.random_network(prob, hidden=32, seed=4, eps=0.1)
    tr = qmc.QMC(N, 16, 99, ND)
    tr.load_schedule(prob)
    tr.set_mlp(net)
    tr.init_populations(P.rho_basis(0))
    feat, target, weight = T.collect_events(tr, DT, STEPS, 20, 4096)
    params = torch.tensor(T.pack(net), device="cuda")
    losses = T.train(tr, params, feat, target, weight, 600, lr=3e-3)
    tg = target.cpu().numpy().astype(np.float64)
    w = weight.cpu().numpy().astype(np.float64)
    ent = float((w * -(np.where(tg > 0, tg * np.log(np.where(tg > 0, tg, 1.0)), 0.0)).sum(axis=0)).sum() / w.sum())
    assert losses[-1] - ent < 0.02 * (losses[0] - ent), (losses[0], losses[-1], ent)

    sd = {}
    for name, mode, p in (("exact", qmc.PROPOSAL_EXACT, None), ("untrained", qmc.PROPOSAL_LEARNED, None),
                          ("trained", qmc.PROPOSAL_LEARNED, params)):
        F = _final_fidelity(prob, net, mode, p)
        sd[name] = F.std(ddof=1)
        assert abs(F.mean() - 0.76) < 0.05, (name, F.mean())
    print("fidelity std over vectors:", {k: round(float(v), 4) for k, v in sd.items()})
    assert sd["trained"] < 0.8 * sd["untrained"], sd
    assert sd["trained"] < 1.3 * sd["exact"], sd
