"""FP64 reference of the learned proposal's training (the library's
extension of the spawn step; not in the paper).

TEST INFRASTRUCTURE ONLY (see the package docstring): plain numpy, float64
unless a value is defined as float32, no blocking or fusion.

Training events.  A logged event is one parent record of N(t), sampled at
record indices r_e = floor(e K / E) of the vectors' records taken in vector
order (all K records when K <= E).  For the source |x><y| of that record:

* features: the n bits of x, the n bits of y (1.0 / 0.0) and float32(t);
* present outputs: the destinations whose static weight (a bound on
  |Re L| + |Im L|, see ``OracleProblem.static``) is positive and that have an
  output of the network; the others get target -1;
* target of a present output: the heat-bath share w_k / W with
  w_k = |Re q_k| + |Im q_k| of the quantised exact column element of dt L(t)
  at that destination (0 where the column has none) and W the sum over the
  present outputs, evaluated as float32(float64(w_k) / float64(W));
* weight: float32(|re| + |im|) of the parent, 0 when W = 0.

Loss.  With the network of the learned proposal (inputs -> ReLU -> ReLU ->
logits) and q = softmax of the logits over the event's present outputs,

    loss = sum_e omega_e CE_e / sum_e omega_e,
    CE_e = -sum_{g present} p_eg log q_eg,

the cross-entropy against the heat-bath shares p (whose minimum puts q at
the exact |L|-weighted choice of the plain method).  Its gradient is the
plain backpropagation of that expression (ReLU derivative 0 at 0).
"""
import numpy as np


def sample_indices(K: int, E: int) -> np.ndarray:
    """Record index of each event: floor(e K / E), or every record."""
    if K <= E:
        return np.arange(K, dtype=np.int64)
    return (np.arange(E, dtype=np.int64) * K) // E


def events(oprob, pops, t: float, dt: float, out_masks, max_events: int):
    """Events from populations ``pops`` (list of (keys, re, im) per vector).
    Returns (feat [I, E], target [G, E], weight [E]) as float32."""
    n = oprob.n
    keys = np.concatenate([np.asarray(p[0], dtype=np.uint64) for p in pops])
    re = np.concatenate([np.asarray(p[1], dtype=np.int64) for p in pops])
    im = np.concatenate([np.asarray(p[2], dtype=np.int64) for p in pops])
    idx = sample_indices(len(keys), max_events)
    E = len(idx)
    out_masks = [int(m) for m in out_masks]
    G, I = len(out_masks), 2 * n + 1
    out_of = {m: g for g, m in enumerate(out_masks)}
    smask, sw = oprob.static(t, dt)
    present_slots = [(int(m), out_of[int(m)]) for m, w in zip(smask, sw) if w > 0 and int(m) in out_of]
    feat = np.zeros((I, E), dtype=np.float32)
    target = np.full((G, E), -1.0, dtype=np.float32)
    weight = np.zeros(E, dtype=np.float32)
    ymask = (1 << n) - 1
    for e, r in enumerate(idx):
        key = int(keys[r])
        x, y = key >> n, key & ymask
        for i in range(n):
            feat[i, e] = float((x >> i) & 1)
            feat[n + i, e] = float((y >> i) & 1)
        feat[2 * n, e] = np.float32(t)
        cm, cre, cim = oprob.column(x, y, t, dt)
        col = {int(m): abs(int(a)) + abs(int(b)) for m, a, b in zip(cm, cre, cim)}
        wk = [(g, col.get(m, 0)) for m, g in present_slots]
        W = sum(w for _, w in wk)
        for g, w in wk:
            target[g, e] = np.float32(np.float64(w) / np.float64(W)) if W > 0 else np.float32(0.0)
        if W > 0:
            weight[e] = np.float32(abs(int(re[r])) + abs(int(im[r])))
    return feat, target, weight


def split_params(flat, I: int, H: int, G: int) -> dict:
    """The packed parameter vector (w1, b1, w2, b2, w3, b3) as arrays."""
    flat = np.asarray(flat, dtype=np.float64)
    shapes = [("w1", (H, I)), ("b1", (H,)), ("w2", (H, H)), ("b2", (H,)), ("w3", (G, H)), ("b3", (G,))]
    out, o = {}, 0
    for name, shp in shapes:
        size = int(np.prod(shp))
        out[name] = flat[o:o + size].reshape(shp)
        o += size
    assert o == flat.size
    return out


def pack(d: dict) -> np.ndarray:
    return np.concatenate([np.asarray(d[k], dtype=np.float64).ravel() for k in ("w1", "b1", "w2", "b2", "w3", "b3")])


def loss_grad(params: dict, feat, target, weight):
    """Loss and gradient (dict like ``params``) in float64."""
    X = np.asarray(feat, dtype=np.float64)            # [I, E]
    T = np.asarray(target, dtype=np.float64)          # [G, E]
    w = np.asarray(weight, dtype=np.float64)          # [E]
    W1, b1, W2, b2, W3, b3 = (params[k] for k in ("w1", "b1", "w2", "b2", "w3", "b3"))
    a1 = W1 @ X + b1[:, None]
    h1 = np.where(a1 > 0, a1, 0.0)
    a2 = W2 @ h1 + b2[:, None]
    h2 = np.where(a2 > 0, a2, 0.0)
    z = W3 @ h2 + b3[:, None]                         # [G, E]
    present = T >= 0
    p = np.where(present, T, 0.0)
    zm = np.where(present, z, -np.inf)
    m = zm.max(axis=0)
    m = np.where(np.isfinite(m), m, 0.0)
    ex = np.where(present, np.exp(zm - m), 0.0)
    S = ex.sum(axis=0)
    Ssafe = np.where(S > 0, S, 1.0)
    q = ex / Ssafe
    logq = np.where(present, z - m - np.log(Ssafe), 0.0)
    ce = -(p * logq).sum(axis=0)                      # [E]
    wsum = w.sum()
    om = w / wsum if wsum > 0 else np.zeros_like(w)
    loss = float((om * ce).sum())
    sp = p.sum(axis=0)
    dz = np.where(present, om * (sp * q - p), 0.0)    # d loss / d z
    g = {"w3": dz @ h2.T, "b3": dz.sum(axis=1)}
    dh2 = (W3.T @ dz) * (a2 > 0)
    g["w2"] = dh2 @ h1.T
    g["b2"] = dh2.sum(axis=1)
    dh1 = (W2.T @ dh2) * (a1 > 0)
    g["w1"] = dh1 @ X.T
    g["b1"] = dh1.sum(axis=1)
    return loss, g


# ---------------------------------------------------------------------------
# The tensor-core proposal's network: bf16 weights and activations, GELU.
# ---------------------------------------------------------------------------
def bf16(x) -> np.ndarray:
    """float32 values rounded to bfloat16 (nearest, ties to even), as float64."""
    a = np.asarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    r = ((a + np.uint64(0x7FFF) + ((a >> np.uint64(16)) & np.uint64(1))) >> np.uint64(16)) << np.uint64(16)
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def gelu(x):
    """GELU in its tanh form, 0.5 x (1 + tanh(sqrt(2/pi) (x + 0.044715 x^3)))."""
    return 0.5 * x * (1.0 + np.tanh(np.sqrt(2.0 / np.pi) * (x + 0.044715 * x ** 3)))


def gelu_prime(x):
    u = np.sqrt(2.0 / np.pi) * (x + 0.044715 * x ** 3)
    th = np.tanh(u)
    return 0.5 * (1.0 + th) + 0.5 * x * (1.0 - th * th) * np.sqrt(2.0 / np.pi) * (1.0 + 3 * 0.044715 * x * x)


def loss_grad_tc(params: dict, feat, target, weight, round_bf16: bool = True):
    """Loss and gradient of the tensor-core proposal's network in float64:
    inputs -> GELU (tanh form) -> GELU -> logits, the weights, the input t and both hidden
    activations rounded to bf16 where the tensor cores take them (the rounding
    passes gradients through unchanged); the same masked weighted
    cross-entropy as ``loss_grad``.  round_bf16=False gives the smooth
    network (for finite differences)."""
    q16 = bf16 if round_bf16 else (lambda v: np.asarray(v, dtype=np.float64))
    X = np.asarray(feat, dtype=np.float64).copy()
    X[-1] = q16(X[-1])                                # t enters as bf16
    T = np.asarray(target, dtype=np.float64)
    w = np.asarray(weight, dtype=np.float64)
    W1, W2, W3 = (q16(params[k]) for k in ("w1", "w2", "w3"))
    b1, b2, b3 = (np.asarray(params[k], dtype=np.float64) for k in ("b1", "b2", "b3"))
    a1 = W1 @ X + b1[:, None]
    h1 = q16(gelu(a1))
    a2 = W2 @ h1 + b2[:, None]
    h2 = q16(gelu(a2))
    z = W3 @ h2 + b3[:, None]
    present = T >= 0
    p = np.where(present, T, 0.0)
    zm = np.where(present, z, -np.inf)
    m = zm.max(axis=0)
    m = np.where(np.isfinite(m), m, 0.0)
    ex = np.where(present, np.exp(zm - m), 0.0)
    S = ex.sum(axis=0)
    Ssafe = np.where(S > 0, S, 1.0)
    q = ex / Ssafe
    logq = np.where(present, z - m - np.log(Ssafe), 0.0)
    ce = -(p * logq).sum(axis=0)
    wsum = w.sum()
    om = w / wsum if wsum > 0 else np.zeros_like(w)
    loss = float((om * ce).sum())
    sp = p.sum(axis=0)
    dz = np.where(present, om * (sp * q - p), 0.0)
    g = {"w3": dz @ h2.T, "b3": dz.sum(axis=1)}
    da2 = (W3.T @ dz) * gelu_prime(a2)
    g["w2"] = da2 @ h1.T
    g["b2"] = da2.sum(axis=1)
    da1 = (W2.T @ da2) * gelu_prime(a1)
    g["w1"] = da1 @ X.T
    g["b1"] = da1.sum(axis=1)
    return loss, g
