"""Dense FP64 reference for tiny n (test infrastructure only).

* ``liouvillian(prob, t)`` builds the D^2 x D^2 matrix of Eq. (2) with Kronecker
  products (column vectorisation, vec(A rho B) = (B^T kron A) vec(rho)):
      L = -i I(x)H + i H^T(x)I + sum_k gamma_k (L_k^* (x) L_k
          - 1/2 I (x) L_k^dag L_k - 1/2 (L_k^dag L_k)^T (x) I).
  Eq. (2) prints L_k (x) L_k and L_k^dag L_k (x) I; those agree with the forms
  above for real L_k (sigma^-, sigma^z), which are the paper's operators.
* ``euler`` / ``ab2`` run the deterministic recursions of the End Matter
  (simulation methodology) on the same time grid as the walker method; since
  every spawn is unbiased and annihilation is exact integer addition, the
  expectation of N(t) / N^diag equals these recursions.
"""
from __future__ import annotations

import math

import numpy as np

_I = np.eye(2, dtype=np.complex128)
_X = np.array([[0, 1], [1, 0]], dtype=np.complex128)
_Y = np.array([[0, -1j], [1j, 0]], dtype=np.complex128)
_Z = np.array([[1, 0], [0, -1]], dtype=np.complex128)


def pauli_matrix(n: int, xm: int, zm: int) -> np.ndarray:
    """Matrix of a Pauli string; qubit q is bit q of the basis index."""
    m = np.ones((1, 1), dtype=np.complex128)
    for q in reversed(range(n)):
        xb, zb = (xm >> q) & 1, (zm >> q) & 1
        s = _Y if (xb and zb) else (_X if xb else (_Z if zb else _I))
        m = np.kron(m, s)
    return m


def rate_value(prob, rid: int, t: float) -> float:
    kind, a, b, c = prob.rates[rid]
    return a * math.cos(b * t + c) if kind == 1 else a


def window_on(prob, wid: int, t: float) -> bool:
    if wid < 0:
        return True
    t0, t1 = prob.windows[wid]
    return t0 <= t < t1


def hamiltonian(prob, t: float) -> np.ndarray:
    D = 1 << prob.n
    H = np.zeros((D, D), dtype=np.complex128)
    for h, xm, zm, rid, wid in prob.ham:
        if window_on(prob, wid, t):
            H += h * rate_value(prob, rid, t) * pauli_matrix(prob.n, xm, zm)
    return H


def lindblad_ops(prob, t: float):
    D = 1 << prob.n
    out = []
    for ops, rid, wid in prob.lind:
        if not window_on(prob, wid, t):
            continue
        L = np.zeros((D, D), dtype=np.complex128)
        for coef, xm, zm in ops:
            L += coef * pauli_matrix(prob.n, xm, zm)
        out.append((rate_value(prob, rid, t), L))
    return out


def liouvillian(prob, t: float) -> np.ndarray:
    """Eq. (2) as a dense matrix acting on column-vectorised rho."""
    D = 1 << prob.n
    eye = np.eye(D, dtype=np.complex128)
    H = hamiltonian(prob, t)
    L = -1j * np.kron(eye, H) + 1j * np.kron(H.T, eye)
    for g, Lk in lindblad_ops(prob, t):
        LdL = Lk.conj().T @ Lk
        L += g * (np.kron(Lk.conj(), Lk) - 0.5 * np.kron(eye, LdL) - 0.5 * np.kron(LdL.T, eye))
    return L


def vec(rho: np.ndarray) -> np.ndarray:
    return rho.reshape(-1, order="F")


def unvec(v: np.ndarray, D: int) -> np.ndarray:
    return v.reshape((D, D), order="F")


def rho_from_entries(n: int, entries) -> np.ndarray:
    D = 1 << n
    rho = np.zeros((D, D), dtype=np.complex128)
    for x, y, re, im in entries:
        rho[x, y] += re + 1j * im
    return rho


def evolve(prob, rho0: np.ndarray, dt: float, nsteps: int, integrator: str = "ab2",
           t0: float = 0.0, record=None) -> np.ndarray:
    """Deterministic Euler / AB2 recursion with L taken at the left end of each
    step; AB2 starts with one Euler step.  ``record(k, rho)`` is called after
    every step if given."""
    D = rho0.shape[0]
    v = vec(rho0).astype(np.complex128)
    prev_term = None
    cache = {}

    def Lof(t):
        if t not in cache:
            cache[t] = liouvillian(prob, t)
        return cache[t]

    for k in range(nsteps):
        t = t0 + k * dt
        cur_term = Lof(t) @ v
        if integrator == "ab2" and prev_term is not None:
            v_new = v + dt * (1.5 * cur_term - 0.5 * prev_term)
        else:
            v_new = v + dt * cur_term
        prev_term = cur_term
        v = v_new
        if record is not None:
            record(k, unvec(v, D))
    return unvec(v, D)


def fidelity(rho: np.ndarray, psi: dict) -> float:
    D = rho.shape[0]
    vecpsi = np.zeros(D, dtype=np.complex128)
    for x, a in psi.items():
        vecpsi[x] = a
    vecpsi /= np.linalg.norm(vecpsi)
    return float(abs(vecpsi.conj() @ rho @ vecpsi))


def evolve_operators(prob, rho0: np.ndarray, dt: float, nsteps: int, integrator: str = "ab2",
                     t0: float = 0.0, record=None) -> np.ndarray:
    """The same Euler / AB2 recursion as ``evolve`` with L(t) applied to rho
    as operators, L(rho) = -i[H, rho] + sum_k gamma_k (L_k rho L_k^dag -
    {L_k^dag L_k, rho} / 2) (Eq. (1)), without forming the D^2 x D^2 matrix:
    for n up to about 10 qubits.  H and the L_k are rebuilt only when the set
    of active pulse windows or the rates change."""
    cache = {}

    def ops(t):
        key = (tuple(window_on(prob, w, t) for w in range(len(prob.windows))),
               tuple(rate_value(prob, r, t) for r in range(len(prob.rates))))
        if key not in cache:
            H = hamiltonian(prob, t)
            Ls = [(g, Lk, Lk.conj().T, Lk.conj().T @ Lk) for g, Lk in lindblad_ops(prob, t)]
            cache.clear()
            cache[key] = (H, Ls)
        return cache[key]

    def apply(t, rho):
        H, Ls = ops(t)
        out = -1j * (H @ rho - rho @ H)
        for g, Lk, Ld, LdL in Ls:
            out += g * (Lk @ rho @ Ld - 0.5 * (LdL @ rho + rho @ LdL))
        return out

    rho = rho0.astype(np.complex128)
    prev_term = None
    for k in range(nsteps):
        t = t0 + k * dt
        cur_term = apply(t, rho)
        if integrator == "ab2" and prev_term is not None:
            rho = rho + dt * (1.5 * cur_term - 0.5 * prev_term)
        else:
            rho = rho + dt * cur_term
        prev_term = cur_term
        if record is not None:
            record(k, rho)
    return rho
