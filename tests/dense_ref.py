"""Dense brute-force route used only to pin the oracle (n <= 6).

Independent of oracle.c: gate matrices come from scipy's matrix exponential of the
Pauli generators (R_sigma(t) = expm(-i t sigma / 2), App. A with alpha = -1/2), U3
from its decomposition e^{i(f+l)/2} RZ(f) RY(t) RZ(l), entanglers from projectors,
and every operator is lifted to the full space by Kronecker products.  Qubit q is
bit q of the index, so the rightmost Kronecker factor is qubit 0.
"""
from __future__ import annotations

import numpy as np
from scipy.linalg import expm

I2 = np.eye(2, dtype=complex)
X = np.array([[0, 1], [1, 0]], dtype=complex)
Y = np.array([[0, -1j], [1j, 0]], dtype=complex)
Z = np.array([[1, 0], [0, -1]], dtype=complex)
P0 = np.array([[1, 0], [0, 0]], dtype=complex)
P1 = np.array([[0, 0], [0, 1]], dtype=complex)
PAULI = {"I": I2, "X": X, "Y": Y, "Z": Z}


def rot(sigma: np.ndarray, t: float) -> np.ndarray:
    return expm(-0.5j * t * sigma)


def u3(t: float, f: float, l: float) -> np.ndarray:
    return np.exp(0.5j * (f + l)) * rot(Z, f) @ rot(Y, t) @ rot(Z, l)


def lift(ops: dict, n: int) -> np.ndarray:
    """Kronecker product with ops[q] on qubit q (identity elsewhere)."""
    m = np.array([[1.0 + 0j]])
    for q in reversed(range(n)):
        m = np.kron(m, ops.get(q, I2))
    return m


def gate_unitary(gate, theta, n: int, shift=None) -> np.ndarray:
    kind, q0, q1, ps = gate
    ang = [theta[p] if p >= 0 else 0.0 for p in ps]
    if shift is not None:
        ang[shift[0]] += shift[1]
    if kind == "RX":
        return lift({q0: rot(X, ang[0])}, n)
    if kind == "RY":
        return lift({q0: rot(Y, ang[0])}, n)
    if kind == "RZ":
        return lift({q0: rot(Z, ang[0])}, n)
    if kind == "U3":
        return lift({q0: u3(*ang)}, n)
    if kind == "CNOT":
        return lift({q0: P0}, n) + lift({q0: P1, q1: X}, n)
    if kind == "CZ":
        return lift({}, n) - 2 * lift({q0: P1, q1: P1}, n)
    if kind in GENERATED:
        return expm(-1j * ang[0] * generator(gate, n))
    raise ValueError(kind)


# Gates built as expm(-i t G) from a Hermitian generator G on the full space (App. A's
# controlled construction is not used here): controlled rotations G = (sigma_t / 2) x
# |1><1|_c, PHASE G = -|1><1|, CPHASE G = -|11><11|.
GENERATED = ("CRX", "CRY", "CRZ", "PHASE", "CPHASE")


def generator(gate, n: int) -> np.ndarray:
    kind, q0, q1, _ps = gate
    if kind in ("CRX", "CRY", "CRZ"):
        sigma = {"CRX": X, "CRY": Y, "CRZ": Z}[kind]
        return 0.5 * lift({q0: P1, q1: sigma}, n)
    if kind == "PHASE":
        return -lift({q0: P1}, n)
    if kind == "CPHASE":
        return -lift({q0: P1, q1: P1}, n)
    raise ValueError(kind)


def gradient_generator(n: int, gates, theta, n_params: int, terms) -> np.ndarray:
    """dE/dtheta by inserting dU/dt = -i G U in place of each one-parameter gate built
    from a generator (rotations use G = sigma/2): exact, no shift rule involved."""
    h = hamiltonian(terms, n)
    psi = state(n, gates, theta)
    g = np.zeros(n_params)
    gens = {"RX": X, "RY": Y, "RZ": Z}
    for i, gate in enumerate(gates):
        kind, q0, _q1, ps = gate
        if kind in gens:
            G = 0.5 * lift({q0: gens[kind]}, n)
        elif kind in GENERATED:
            G = generator(gate, n)
        else:
            if any(p >= 0 for p in ps):
                raise ValueError(f"no generator route for {kind}")
            continue
        mu = np.zeros(1 << n, dtype=complex)
        mu[0] = 1
        for k, gk in enumerate(gates):
            u = gate_unitary(gk, theta, n)
            mu = (-1j * G @ u @ mu) if k == i else (u @ mu)
        g[ps[0]] += 2 * np.real(psi.conj() @ h @ mu)
    return g


def hamiltonian(terms, n: int) -> np.ndarray:
    h = np.zeros((1 << n, 1 << n), dtype=complex)
    for c, ops in terms:
        h += c * lift({q: PAULI[l] for q, l in ops}, n)
    return h


def state(n: int, gates, theta, shift_at=None) -> np.ndarray:
    psi = np.zeros(1 << n, dtype=complex)
    psi[0] = 1
    for i, g in enumerate(gates):
        sh = shift_at[1:] if (shift_at is not None and shift_at[0] == i) else None
        psi = gate_unitary(g, theta, n, sh) @ psi
    return psi


def energy(n: int, gates, theta, terms, shift_at=None) -> float:
    psi = state(n, gates, theta, shift_at)
    return float(np.real(psi.conj() @ hamiltonian(terms, n) @ psi))


def gradient_shift(n: int, gates, theta, n_params: int, terms) -> np.ndarray:
    """Per-occurrence parameter shift on the dense route."""
    g = np.zeros(n_params)
    for i, (kind, _q0, _q1, ps) in enumerate(gates):
        for j, p in enumerate(ps):
            if p < 0:
                continue
            ep = energy(n, gates, theta, terms, (i, j, np.pi / 2))
            em = energy(n, gates, theta, terms, (i, j, -np.pi / 2))
            g[p] += 0.5 * (ep - em)
    return g


def gradient_fd(n: int, gates, theta, n_params: int, terms, delta: float = 1e-5) -> np.ndarray:
    """Central finite differences on the dense route (Eq. 2, symmetric form)."""
    g = np.zeros(n_params)
    th = np.array(theta, dtype=float)
    for p in range(n_params):
        tp = th.copy(); tp[p] += delta
        tm = th.copy(); tm[p] -= delta
        g[p] = (energy(n, gates, tp, terms) - energy(n, gates, tm, terms)) / (2 * delta)
    return g


def operator(terms, n: int) -> np.ndarray:
    """Dense operator of a Pauli sum with complex coefficients (non-Hermitian in general)."""
    a = np.zeros((1 << n, 1 << n), dtype=complex)
    for c, ops in terms:
        a += complex(c) * lift({q: PAULI[l] for q, l in ops}, n)
    return a


def expectation_complex(n: int, gates, theta, terms) -> complex:
    psi = state(n, gates, theta)
    return complex(psi.conj() @ operator(terms, n) @ psi)


def gradient_fd_complex(n: int, gates, theta, n_params: int, terms, delta: float = 1e-5) -> np.ndarray:
    """Central differences of the complex expectation (real and imaginary parts at once)."""
    g = np.zeros(n_params, dtype=complex)
    th = np.array(theta, dtype=float)
    for p in range(n_params):
        tp = th.copy(); tp[p] += delta
        tm = th.copy(); tm[p] -= delta
        g[p] = (expectation_complex(n, gates, tp, terms) - expectation_complex(n, gates, tm, terms)) / (2 * delta)
    return g
