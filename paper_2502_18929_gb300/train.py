"""Training of the learned proposal's network on the method's own spawn
statistics (the library's extension; not in the paper).

Host orchestration only: events, loss, gradient and the Adam update all run
in the library's CUDA kernels (qmc_learn_*); this module loops over them.

The network learns the plain method's heat-bath destination choice (share
|Re L| + |Im L| of each destination): at its optimum the learned proposal's
walker counts are Bernoulli like the plain method's, so training removes the
extra variance an untrained proposal adds (counts above one).  It cannot beat
the plain method's per-walker variance, which is already minimal.
"""
from __future__ import annotations

import numpy as np

PARAM_ORDER = ("w1", "b1", "w2", "b2", "w3", "b3")


def pack(net: dict) -> np.ndarray:
    """Packed float32 parameters (w1, b1, w2, b2, w3, b3) of a network dict."""
    return np.concatenate([np.asarray(net[k], dtype=np.float32).ravel() for k in PARAM_ORDER])


def unpack(flat, net: dict) -> dict:
    """A network dict like ``net`` with the packed parameters ``flat``."""
    flat = np.asarray(flat, dtype=np.float32)
    out, o = dict(net), 0
    for k in PARAM_ORDER:
        shp = np.shape(net[k])
        size = int(np.prod(shp))
        out[k] = flat[o:o + size].reshape(shp).copy()
        o += size
    assert o == flat.size
    return out


def collect_events(sim, dt: float, nsteps: int, every: int, max_events: int):
    """Step ``sim`` (its current proposal) ``nsteps`` times and log training
    events from N(t) every ``every`` steps.  Returns the event sets joined
    along the event axis (feat, target, weight) as CUDA tensors."""
    import torch
    feats, targets, weights = [], [], []
    done = 0
    while done < nsteps:
        f, t, w, ne = sim.learn_events(dt, max_events)
        feats.append(f[:, :ne])
        targets.append(t[:, :ne])
        weights.append(w[:ne])
        k = min(every, nsteps - done)
        sim.step(dt, k)
        done += k
    return (torch.cat(feats, dim=1).contiguous(), torch.cat(targets, dim=1).contiguous(),
            torch.cat(weights).contiguous())


def train(sim, params, feat, target, weight, steps: int, lr: float = 3e-3):
    """Full-batch Adam on the events; returns the loss before each step.
    ``params`` (CUDA float32, packed) is updated in place."""
    import torch
    m = torch.zeros_like(params)
    v = torch.zeros_like(params)
    E = feat.shape[1]
    losses = []
    for t in range(1, steps + 1):
        loss, grad = sim.learn_grad(params, feat, target, weight, E)
        losses.append(loss)
        sim.learn_adam(params, grad, m, v, t, lr)
    return losses
