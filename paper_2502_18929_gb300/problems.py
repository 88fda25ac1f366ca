"""Problem descriptions and seeded synthetic inputs.

This module only *describes* master equations and initial populations; it holds
none of the method's arithmetic (no Liouvillian expansion, no sampling).  Both
the CUDA path and the CPU oracle consume the same description.

Conventions
-----------
* Qubit ``q`` is bit ``q`` of a basis index ``x`` (``x = sum_q x_q 2**q``).
* A Pauli string is a pair of bit masks ``(xm, zm)``: qubit ``q`` carries
  ``I`` (0,0), ``X`` (1,0), ``Z`` (0,1) or the Hermitian ``Y`` (1,1).
* The master equation is Eq. (1):
  ``drho/dt = -i[H(t), rho] + 1/2 sum_k gamma_k(t) D[L_k] rho`` with
  ``D[L] rho = 2 L rho L^dag - {L^dag L, rho}``.
  ``H(t) = sum_j h_j r_j(t) w_j(t) P_j`` and each ``L_k = sum_a l_a P_a``.
* Rates: kind 0 = constant ``a``; kind 1 = ``a * cos(b * t + c)``.
* Windows: ``[t0, t1)``; window id -1 means "always on".
* A density-matrix element ``rho_xy`` lives at the packed key ``(x << n) | y``.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

RATE_CONST = 0
RATE_COS = 1
ALWAYS = -1


def pauli(spec: dict[int, str]) -> tuple[int, int]:
    """Return ``(xm, zm)`` for a Pauli string given as ``{qubit: 'X'|'Y'|'Z'}``."""
    xm = zm = 0
    for q, letter in spec.items():
        letter = letter.upper()
        if letter in ("X", "Y"):
            xm |= 1 << q
        if letter in ("Z", "Y"):
            zm |= 1 << q
        if letter not in ("I", "X", "Y", "Z"):
            raise ValueError(f"bad Pauli letter {letter!r}")
    return xm, zm


@dataclass
class Problem:
    """A time-local master equation over ``n`` qubits (Eq. (1))."""

    n: int
    ham: list = field(default_factory=list)      # (h, xm, zm, rate_id, window_id)
    lind: list = field(default_factory=list)     # ([(coef complex, xm, zm)], rate_id, window_id)
    rates: list = field(default_factory=list)    # (kind, a, b, c)
    windows: list = field(default_factory=list)  # (t0, t1)
    name: str = ""
    t_end: float = 0.0

    # -- construction helpers -------------------------------------------------
    def rate(self, kind: int, a: float, b: float = 0.0, c: float = 0.0) -> int:
        self.rates.append((int(kind), float(a), float(b), float(c)))
        return len(self.rates) - 1

    def window(self, t0: float, t1: float) -> int:
        self.windows.append((float(t0), float(t1)))
        return len(self.windows) - 1

    def add_h(self, h: float, spec: dict[int, str], rate: int, window: int = ALWAYS):
        xm, zm = pauli(spec)
        self.ham.append((float(h), xm, zm, int(rate), int(window)))

    def add_lindblad(self, ops: list, rate: int, window: int = ALWAYS):
        """``ops`` is a list of ``(complex coefficient, {qubit: letter})``."""
        terms = []
        for coef, spec in ops:
            xm, zm = pauli(spec)
            terms.append((complex(coef), xm, zm))
        self.lind.append((terms, int(rate), int(window)))

    # -- flat arrays for the C interfaces ------------------------------------
    def arrays(self) -> dict:
        h = np.array([t[0] for t in self.ham], dtype=np.float64)
        hx = np.array([t[1] for t in self.ham], dtype=np.uint64)
        hz = np.array([t[2] for t in self.ham], dtype=np.uint64)
        hr = np.array([t[3] for t in self.ham], dtype=np.int32)
        hw = np.array([t[4] for t in self.ham], dtype=np.int32)
        lstart, lcount, lrate, lwin = [], [], [], []
        lre, lim, lx, lz = [], [], [], []
        for ops, r, w in self.lind:
            lstart.append(len(lre))
            lcount.append(len(ops))
            lrate.append(r)
            lwin.append(w)
            for coef, xm, zm in ops:
                lre.append(coef.real)
                lim.append(coef.imag)
                lx.append(xm)
                lz.append(zm)
        return dict(
            h=h, hx=hx, hz=hz, hrate=hr, hwin=hw,
            lstart=np.array(lstart, dtype=np.int32), lcount=np.array(lcount, dtype=np.int32),
            lrate=np.array(lrate, dtype=np.int32), lwin=np.array(lwin, dtype=np.int32),
            lre=np.array(lre, dtype=np.float64), lim=np.array(lim, dtype=np.float64),
            lx=np.array(lx, dtype=np.uint64), lz=np.array(lz, dtype=np.uint64),
            rkind=np.array([r[0] for r in self.rates], dtype=np.int32),
            ra=np.array([r[1] for r in self.rates], dtype=np.float64),
            rb=np.array([r[2] for r in self.rates], dtype=np.float64),
            rc=np.array([r[3] for r in self.rates], dtype=np.float64),
            wt0=np.array([w[0] for w in self.windows], dtype=np.float64),
            wt1=np.array([w[1] for w in self.windows], dtype=np.float64),
        )

    def boundaries(self, t_end: float | None = None) -> list[float]:
        """Sorted window edges inside ``[0, t_end]`` (segment edges for a run)."""
        t_end = self.t_end if t_end is None else t_end
        edges = {0.0, float(t_end)}
        for t0, t1 in self.windows:
            for e in (t0, t1):
                if 0.0 < e < t_end:
                    edges.add(float(e))
        return sorted(edges)


# ---------------------------------------------------------------------------
# Noise channels used throughout the paper's circuits (transmon model):
# amplitude damping L = sigma^- = |0><1| = (X + iY)/2 and dephasing L = Z.
# ---------------------------------------------------------------------------

def add_local_noise(p: Problem, gamma1: float, gamma_phi: float, x_basis: bool = False,
                    rate_kind: int = RATE_CONST, omega1: float = 0.0, omega_phi: float = 0.0):
    """Per-qubit amplitude damping (rate gamma1) and dephasing (rate gamma_phi).

    With ``x_basis`` every operator is conjugated by Hadamards (X <-> Z, Y -> -Y),
    which is how a ``|+>``-type initial state is kept sparse.
    With ``rate_kind == RATE_COS`` the rates are ``gamma * cos(omega t)`` (negative
    half-periods are non-Markovian).
    """
    r1 = p.rate(rate_kind, gamma1, omega1 if rate_kind == RATE_COS else 0.0)
    rp = p.rate(rate_kind, gamma_phi, omega_phi if rate_kind == RATE_COS else 0.0)
    for q in range(p.n):
        if gamma1 != 0.0:
            if x_basis:
                # H sigma^- H = (Z - iY)/2
                p.add_lindblad([(0.5, {q: "Z"}), (-0.5j, {q: "Y"})], r1)
            else:
                p.add_lindblad([(0.5, {q: "X"}), (0.5j, {q: "Y"})], r1)
        if gamma_phi != 0.0:
            p.add_lindblad([(1.0, {q: "X" if x_basis else "Z"})], rp)


def add_hadamard_pulse(p: Problem, q: int, t0: float, t1: float):
    """Square pulse whose propagator over ``[t0, t1)`` is the Hadamard gate.

    Generator (pi/2)(I - (X+Z)/sqrt 2) / (t1 - t0); the identity part drops out of
    the commutator, so only the X and Z parts are kept.
    """
    dur = t1 - t0
    w = p.window(t0, t1)
    one = p.rate(RATE_CONST, 1.0)
    amp = -(math.pi / 2.0) / math.sqrt(2.0) / dur
    p.add_h(amp, {q: "X"}, one, w)
    p.add_h(amp, {q: "Z"}, one, w)


def add_cnot_pulse(p: Problem, c: int, t: int, t0: float, t1: float):
    """Square pulse with generator (pi/4)(1 - Z_c)(1 - X_t) / (t1 - t0).

    exp(-i pi Proj) with Proj = |1><1|_c (x) |-><-|_t is exactly CNOT.  The
    identity part is dropped (it commutes with everything).
    """
    dur = t1 - t0
    w = p.window(t0, t1)
    one = p.rate(RATE_CONST, 1.0)
    a = (math.pi / 4.0) / dur
    p.add_h(-a, {c: "Z"}, one, w)
    p.add_h(-a, {t: "X"}, one, w)
    p.add_h(a, {c: "Z", t: "X"}, one, w)


def ghz_circuit(n: int, gamma1: float = 0.01, gamma_phi: float = 0.02, pulse: float = 1.0,
                rate_kind: int = RATE_CONST, omega1: float = 0.0, omega_phi: float = 0.0) -> Problem:
    """GHZ preparation: Hadamard on q0, then CNOT(q_i -> q_{i+1}); each gate is a
    square pulse of duration ``pulse`` (Fig. 1(d)), under local noise."""
    p = Problem(n=n, name=f"ghz{n}")
    add_hadamard_pulse(p, 0, 0.0, pulse)
    for i in range(n - 1):
        add_cnot_pulse(p, i, i + 1, (i + 1) * pulse, (i + 2) * pulse)
    add_local_noise(p, gamma1, gamma_phi, rate_kind=rate_kind, omega1=omega1, omega_phi=omega_phi)
    p.t_end = n * pulse
    return p


def dd_ring(n: int = 12, seed: int = 0, gamma_phi: float = 5e-3, gamma1: float = 2e-3,
            width: float = 0.02, tau: float = 1.0, t_end: float = 20.0,
            x_basis: bool = True) -> Problem:
    """Staggered XX dynamical decoupling on a ring with ZZ crosstalk (Fig. 1(c)).

    ``H = sum_i J_i Z_i Z_{i+1}`` (ring), ``J_i ~ U[0.5, 1.5] * 2 pi * 1e-3`` from
    ``seed``.  Even qubits get X pulses at tau/2 + k tau, odd qubits at tau + k tau
    (each a square pi pulse of duration ``width``).  In the X basis (the sparse
    frame for ``|+>^n``) ZZ -> XX and the X pulses become Z pulses.
    """
    rng = np.random.default_rng(seed)
    J = rng.uniform(0.5, 1.5, size=n) * 2.0 * math.pi * 1e-3
    p = Problem(n=n, name=f"dd{n}")
    one = p.rate(RATE_CONST, 1.0)
    zz = "X" if x_basis else "Z"
    for i in range(n):
        p.add_h(float(J[i]), {i: zz, (i + 1) % n: zz}, one)
    amp = math.pi / (2.0 * width)
    letter = "Z" if x_basis else "X"
    k = 0
    while True:
        placed = False
        for q in range(n):
            start = (tau / 2.0 if q % 2 == 0 else tau) + k * tau
            if start + width <= t_end:
                w = p.window(start, start + width)
                p.add_h(amp, {q: letter}, one, w)
                placed = True
        if not placed:
            break
        k += 1
    add_local_noise(p, gamma1, gamma_phi, x_basis=x_basis)
    p.t_end = t_end
    return p


def pure_noise(n: int, gamma1: float, gamma_phi: float, rate_kind: int = RATE_CONST,
               omega1: float = 0.0, omega_phi: float = 0.0) -> Problem:
    p = Problem(n=n, name=f"noise{n}")
    add_local_noise(p, gamma1, gamma_phi, rate_kind=rate_kind, omega1=omega1, omega_phi=omega_phi)
    return p


# ---------------------------------------------------------------------------
# Initial density matrices (sparse) and observable targets
# ---------------------------------------------------------------------------

def _pauli_mat(n: int, xm: int, zm: int) -> np.ndarray:
    """Matrix of a Pauli string (qubit q is bit q of the basis index)."""
    one = {(0, 0): np.eye(2), (1, 0): np.array([[0, 1], [1, 0]]), (0, 1): np.diag([1.0, -1.0]),
           (1, 1): np.array([[0, -1j], [1j, 0]])}
    m = np.ones((1, 1), dtype=np.complex128)
    for q in reversed(range(n)):
        m = np.kron(m, one[((xm >> q) & 1, (zm >> q) & 1)])
    return m


def pauli_terms(M: np.ndarray, n: int, tol: float = 1e-14) -> list:
    """Pauli-string expansion of an operator on n qubits: [(coef, xm, zm)]
    with M = sum coef P (coef = Tr(P M) / 2^n), tiny terms dropped."""
    D = 1 << n
    out = []
    for xm in range(D):
        for zm in range(D):
            c = complex(np.trace(_pauli_mat(n, xm, zm) @ M)) / D
            if abs(c) > tol:
                out.append((c, xm, zm))
    return out


def redfield_two_qubits(omega1: float = 0.25, omega2: float = 0.5, gamma1: float = 1.0, gamma2: float = 4.0,
                        alpha: float = 3.0, kappa: float = 1.0):
    """Two qubits collectively coupled to one bosonic bath, as the Redfield
    master equation Eq. (4) [Non-Markovian dynamics; End Matter on the Redfield
    equation]: drho/dt = -i sum_ij A_ij [s_j^+ s_i^-, rho] + sum_k lambda_k
    D[L_k] rho, with the frequency matrix A of the End Matter (Lamb shifts
    alpha and kappa given as inputs).

    The dissipator comes from the bath's rate matrix over the jump operators
    s_1^-, s_2^- (reading, the paper prints only its eigenvalues):
        G = [[g1 / 2, (g1 + g2) / 4 + i kappa], [(g1 + g2) / 4 - i kappa, g2 / 2]],
    whose eigenvalues are the paper's lambda_k = (g1 + g2) / 4 -/+
    sqrt((g1^2 + g2^2 + 8 kappa^2) / 8) (one of them negative: non-Markovian);
    with G = U diag(lambda) U^dag, L_k = sum_j conj(U_jk) s_j^-, so that
    sum_ij G_ij (s_j rho s_i^dag - {s_i^dag s_j, rho} / 2) = sum_k lambda_k
    (L_k rho L_k^dag - {L_k^dag L_k, rho} / 2).  As the paper does, the problem
    is written in the basis |0~> = |00>, |1~> = L_1^dag |00>, |2~> =
    L_2^dag |00>, |3~> ~ L_2^dag L_1^dag |00> (normalised), basis state b
    stored at index b.  Returns (Problem, info) with info = dict(lam, A, G, V)
    (V: the new basis vectors as columns, in the computational basis)."""
    # qubit q is bit q: s_q^- = |0><1| on qubit q
    sm1 = np.array([[0, 1], [0, 0]], dtype=np.complex128)
    eye = np.eye(2, dtype=np.complex128)
    s = [np.kron(eye, sm1), np.kron(sm1, eye)]
    A = np.array([[omega1 + alpha, alpha + kappa / 2 - 1j * (gamma1 - gamma2) / 8],
                  [alpha + kappa / 2 - 1j * (gamma2 - gamma1) / 8, omega2 + alpha + kappa]])
    H = sum(A[i, j] * s[j].conj().T @ s[i] for i in range(2) for j in range(2))
    G = np.array([[gamma1 / 2, (gamma1 + gamma2) / 4 + 1j * kappa],
                  [(gamma1 + gamma2) / 4 - 1j * kappa, gamma2 / 2]])
    lam, U = np.linalg.eigh(G)
    L = [sum(np.conj(U[j, k]) * s[j] for j in range(2)) for k in range(2)]
    v0 = np.zeros(4, dtype=np.complex128)
    v0[0] = 1.0
    v3 = L[1].conj().T @ L[0].conj().T @ v0
    V = np.stack([v0, L[0].conj().T @ v0, L[1].conj().T @ v0, v3 / np.linalg.norm(v3)], axis=1)
    Ht = V.conj().T @ H @ V
    Lt = [V.conj().T @ Lk @ V for Lk in L]
    p = Problem(2, name="redfield2")
    one = p.rate(RATE_CONST, 1.0)
    for c, xm, zm in pauli_terms(Ht, 2):
        p.ham.append((float(c.real), xm, zm, one, ALWAYS))
    for k in range(2):
        rk = p.rate(RATE_CONST, float(lam[k]))
        p.lind.append((pauli_terms(Lt[k], 2), rk, ALWAYS))
    return p, {"lam": lam, "A": A, "G": G, "V": V}


def rho_basis(x: int = 0) -> list:
    """``|x><x|`` as sparse entries ``(x, y, re, im)``."""
    return [(x, x, 1.0, 0.0)]


def rho_pure(amplitudes: dict[int, complex]) -> list:
    """``|psi><psi|`` for a sparse ``psi`` (normalised here)."""
    norm = math.sqrt(sum(abs(a) ** 2 for a in amplitudes.values()))
    out = []
    for x, ax in sorted(amplitudes.items()):
        for y, ay in sorted(amplitudes.items()):
            v = (ax / norm) * (ay / norm).conjugate()
            if v != 0:
                out.append((x, y, v.real, v.imag))
    return out


def ghz_target(n: int) -> dict[int, complex]:
    return {0: 1.0, (1 << n) - 1: 1.0}


def w_state(n: int) -> dict[int, complex]:
    return {1 << q: 1.0 for q in range(n)}


def spread_population(n: int, count: int, seed: int) -> tuple[np.ndarray, np.ndarray, np.ndarray]:
    """``count`` distinct uniformly random keys over 2n bits, each holding one
    walker of sign +1, -1, +i or -i.  Returns sorted keys and int32 (re, im)."""
    rng = np.random.default_rng(seed)
    bits = 2 * n

    def draw(m):
        if bits >= 64:
            return rng.integers(0, 2**63, size=m, dtype=np.uint64) * np.uint64(2) + \
                rng.integers(0, 2, size=m, dtype=np.uint64)
        return rng.integers(0, 1 << bits, size=m, dtype=np.uint64)

    def distinct(a):
        a = np.sort(a)
        return a[np.concatenate([[True], a[1:] != a[:-1]])] if a.size else a

    keys = distinct(draw(count))
    while keys.size < count:   # duplicates drawn: add more, then keep a uniform subset
        keys = distinct(np.concatenate([keys, draw(count - keys.size + 16)]))
    if keys.size > count:
        keys = np.sort(rng.choice(keys, size=count, replace=False))
    sel = rng.integers(0, 4, size=count)
    re = np.where(sel == 0, 1, np.where(sel == 1, -1, 0)).astype(np.int32)
    im = np.where(sel == 2, 1, np.where(sel == 3, -1, 0)).astype(np.int32)
    return keys, re, im


def spread_population_xy(n: int, count: int, seed: int):
    """``count`` distinct uniformly random states |x><y| of n qubits (any n
    up to 64), each holding one walker of sign +1, -1, +i or -i, in key order
    ((x, y) ascending).  Returns uint64 x, y and int32 (re, im)."""
    rng = np.random.default_rng(seed)
    hi = 1 << n

    def draw(m):
        if n == 64:
            return rng.integers(0, 2**64 - 1, size=m, dtype=np.uint64, endpoint=True)
        return rng.integers(0, hi, size=m, dtype=np.uint64)

    def distinct(x, y):
        o = np.lexsort((y, x))
        x, y = x[o], y[o]
        keep = np.concatenate([[True], (x[1:] != x[:-1]) | (y[1:] != y[:-1])]) if x.size else np.zeros(0, bool)
        return x[keep], y[keep]

    x, y = distinct(draw(count), draw(count))
    while x.size < count:
        m = count - x.size + 16
        x, y = distinct(np.concatenate([x, draw(m)]), np.concatenate([y, draw(m)]))
    if x.size > count:
        pick = np.sort(rng.choice(x.size, size=count, replace=False))
        x, y = x[pick], y[pick]
    sel = rng.integers(0, 4, size=count)
    re = np.where(sel == 0, 1, np.where(sel == 1, -1, 0)).astype(np.int32)
    im = np.where(sel == 2, 1, np.where(sel == 3, -1, 0)).astype(np.int32)
    return x, y, re, im


def destination_masks(prob) -> np.ndarray:
    """Every destination mask (dx << n) | dy that a term of the problem can
    reach (a Pauli string flips the bits of its X part), sorted."""
    n = prob.n
    out = set()
    for h, xm, zm, r, w in prob.ham:
        out.add(int(xm) << n)
        out.add(int(xm))
    for ops, r, w in prob.lind:
        for _, xa, _ in ops:
            for _, xb, _ in ops:
                out.add((int(xa) << n) | int(xb))
                out.add((int(xa) ^ int(xb)) << n)
                out.add(int(xa) ^ int(xb))
    return np.array(sorted(out), dtype=np.uint64)


def random_network(prob, hidden: int = 32, seed: int = 0, eps: float = 0.25, scale: float = 1.0) -> dict:
    """Randomly initialised network of the learned proposal for a problem:
    inputs the n bits of x, the n bits of y and t; one output per
    destination mask (float32, row-major weights)."""
    rng = np.random.default_rng(seed)
    masks = destination_masks(prob)
    I = 2 * prob.n + 1
    f32 = np.float32
    return {
        "out_masks": masks,
        "w1": (rng.standard_normal((hidden, I)) * scale / np.sqrt(I)).astype(f32),
        "b1": (rng.standard_normal(hidden) * 0.1).astype(f32),
        "w2": (rng.standard_normal((hidden, hidden)) * scale / np.sqrt(hidden)).astype(f32),
        "b2": (rng.standard_normal(hidden) * 0.1).astype(f32),
        "w3": (rng.standard_normal((len(masks), hidden)) * scale / np.sqrt(hidden)).astype(f32),
        "b3": (rng.standard_normal(len(masks)) * 0.5).astype(f32),
        "eps": float(eps),
    }
