"""Seeded synthetic workloads: ansatz gate lists, parameter vectors and Pauli-sum
Hamiltonians.

This module only *describes* inputs.  It holds none of the method's arithmetic
(no gate matrices, no state vectors, no Pauli algebra), so both the CUDA path and
the CPU oracle may consume its output without sharing any computation.

Neutral formats
---------------
gate      : (kind, q0, q1, (p0, p1, p2)) with kind in {"RX","RY","RZ","U3","CNOT","CZ",
            "CRX","CRY","CRZ","PHASE","CPHASE"}; q1 = -1 for one-qubit gates; unused
            parameter slots are -1.  For CNOT and the controlled rotations q0 is the
            control and q1 the target.  U3 parameter slots are (theta, phi, lam).
term      : (coef, ((qubit, letter), ...)) with letter in "XYZ"; qubits absent from
            the tuple carry the identity.  Duplicate strings are allowed (they add).

Circuit structure and parameter numbering follow the paper's problem statement
(Sec. 2.2: U = U_P ... U_1 acting on a fixed input state, one parameter per gate
unless a gate carries several, App. B.1).  Parameter indices are assigned in gate
order.  The input state is |0...0>.

Workload recipes (random stream: numpy default_rng(2009_02823 + cfg); theta is drawn
first, U[0, 2pi) in parameter-index order, then any Hamiltonian randomness):

cfg1  n=10, 4 layers of [RY(q), RZ(q) for q=0..n-1; CNOT q->q+1 for q=0..n-2], P=80,
      H = TFIM sum Z_i Z_{i+1} + 1.0 sum X_i (open chain).
cfg2  n=24, 20 layers of the same ansatz (P=960, G=1420),
      H = XXZ periodic sum (X_i X_{i+1} + Y_i Y_{i+1} + 0.5 Z_i Z_{i+1}).
cfg3  n=30, 10 layers of [RY(q), RZ(q) for all q; CZ brickwork], P=600, G=745,
      CZ on (2k, 2k+1) in even layers and (2k+1, 2k+2) in odd layers,
      H = 200 random Pauli strings, weight w ~ U{1..4}, qubits without replacement,
      letters ~ U{X,Y,Z}, coefficients ~ N(0, 1).
cfg4  512 independent circuits, n_b ~ U{12..20}, d_b ~ U{4..16} layers of the cfg1
      ansatz, own theta, TFIM with field h_b ~ U[0.5, 1.5].
cfg5  n=26, 12 layers of [U3(q) for all q; CZ brickwork], P=936, G=462,
      H = TFIM with h = 1.0 (open chain).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

SEED_BASE = 2009_02823

ONE_QUBIT = ("RX", "RY", "RZ", "U3", "PHASE")
TWO_QUBIT = ("CNOT", "CZ")
CONTROLLED = ("CRX", "CRY", "CRZ", "CPHASE")  # two-qubit, one parameter; q0 = control
N_PARAMS_OF = {"RX": 1, "RY": 1, "RZ": 1, "U3": 3, "CNOT": 0, "CZ": 0,
               "CRX": 1, "CRY": 1, "CRZ": 1, "PHASE": 1, "CPHASE": 1}


@dataclass
class Workload:
    """One circuit + parameters + Hamiltonian in the neutral formats above."""

    name: str
    n: int
    gates: list
    n_params: int
    theta: np.ndarray
    terms: list
    meta: dict = field(default_factory=dict)

    @property
    def n_gates(self) -> int:
        return len(self.gates)


class _Builder:
    """Appends gates and hands out parameter indices in gate order."""

    def __init__(self, n: int):
        self.n = n
        self.gates: list = []
        self.n_params = 0

    def rot(self, kind: str, q: int) -> None:
        k = N_PARAMS_OF[kind]
        params = tuple(self.n_params + j for j in range(k)) + (-1,) * (3 - k)
        self.n_params += k
        self.gates.append((kind, q, -1, params))

    def two(self, kind: str, a: int, b: int) -> None:
        self.gates.append((kind, a, b, (-1, -1, -1)))

    def ctrl(self, kind: str, c: int, t: int) -> None:
        self.gates.append((kind, c, t, (self.n_params, -1, -1)))
        self.n_params += 1


def cnot_ladder(b: _Builder) -> None:
    for q in range(b.n - 1):
        b.two("CNOT", q, q + 1)


def cz_brick(b: _Builder, layer: int) -> None:
    start = 0 if layer % 2 == 0 else 1
    for a in range(start, b.n - 1, 2):
        b.two("CZ", a, a + 1)


def hea_ry_rz(n: int, layers: int, entangler: str = "cnot_ladder") -> tuple[list, int]:
    """Hardware-efficient ansatz: per layer RY(q), RZ(q) on every qubit, then entanglers."""
    b = _Builder(n)
    for layer in range(layers):
        for q in range(n):
            b.rot("RY", q)
            b.rot("RZ", q)
        if entangler == "cnot_ladder":
            cnot_ladder(b)
        elif entangler == "cz_brick":
            cz_brick(b, layer)
        else:
            raise ValueError(entangler)
    return b.gates, b.n_params


def u3_brick(n: int, layers: int) -> tuple[list, int]:
    """Per layer U3(q) on every qubit, then the CZ brickwork."""
    b = _Builder(n)
    for layer in range(layers):
        for q in range(n):
            b.rot("U3", q)
        cz_brick(b, layer)
    return b.gates, b.n_params


def tfim(n: int, h: float = 1.0, periodic: bool = False) -> list:
    """sum_i Z_i Z_{i+1} + h sum_i X_i (signs taken literally as '+')."""
    terms = []
    last = n if periodic else n - 1
    for i in range(last):
        terms.append((1.0, ((i, "Z"), ((i + 1) % n, "Z"))))
    for i in range(n):
        terms.append((float(h), ((i, "X"),)))
    return terms


def xxz(n: int, delta: float = 0.5, periodic: bool = True) -> list:
    """sum_i (X_i X_{i+1} + Y_i Y_{i+1} + delta Z_i Z_{i+1})."""
    terms = []
    last = n if periodic else n - 1
    for i in range(last):
        j = (i + 1) % n
        terms.append((1.0, ((i, "X"), (j, "X"))))
        terms.append((1.0, ((i, "Y"), (j, "Y"))))
        terms.append((float(delta), ((i, "Z"), (j, "Z"))))
    return terms


def random_paulis(rng: np.random.Generator, n: int, count: int, wmax: int = 4) -> list:
    """count strings: weight ~ U{1..wmax}, distinct qubits, letters ~ U{X,Y,Z}, coef ~ N(0,1)."""
    terms = []
    for _ in range(count):
        w = int(rng.integers(1, wmax + 1))
        qs = rng.choice(n, size=w, replace=False)
        letters = rng.integers(0, 3, size=w)
        coef = float(rng.standard_normal())
        ops = tuple(sorted((int(q), "XYZ"[int(l)]) for q, l in zip(qs, letters)))
        terms.append((coef, ops))
    return terms


def draw_theta(rng: np.random.Generator, n_params: int) -> np.ndarray:
    return rng.uniform(0.0, 2.0 * math.pi, size=n_params)


def config(cfg: int, n: int | None = None, layers: int | None = None) -> Workload:
    """The cfg-th workload.  n / layers may be overridden to get a smaller case with
    the same structure (the parity tests use this at sizes the oracle finishes in
    seconds); the random stream is the same recipe either way."""
    rng = np.random.default_rng(SEED_BASE + cfg)
    if cfg == 1:
        n = n or 10
        layers = layers or 4
        gates, P = hea_ry_rz(n, layers, "cnot_ladder")
        theta = draw_theta(rng, P)
        terms = tfim(n, 1.0, periodic=False)
        name = f"hea_ry_rz_cnot_n{n}_L{layers}_tfim"
    elif cfg == 2:
        n = n or 24
        layers = layers or 20
        gates, P = hea_ry_rz(n, layers, "cnot_ladder")
        theta = draw_theta(rng, P)
        terms = xxz(n, 0.5, periodic=True)
        name = f"hea_ry_rz_cnot_n{n}_L{layers}_xxz"
    elif cfg == 3:
        n = n or 30
        layers = layers or 10
        gates, P = hea_ry_rz(n, layers, "cz_brick")
        theta = draw_theta(rng, P)
        terms = random_paulis(rng, n, 200, 4)
        name = f"hea_ry_rz_czbrick_n{n}_L{layers}_rand200"
    elif cfg == 5:
        n = n or 26
        layers = layers or 12
        gates, P = u3_brick(n, layers)
        theta = draw_theta(rng, P)
        terms = tfim(n, 1.0, periodic=False)
        name = f"u3_czbrick_n{n}_L{layers}_tfim"
    else:
        raise ValueError(f"no single-circuit workload for cfg={cfg}")
    return Workload(name=name, n=n, gates=gates, n_params=P, theta=theta, terms=terms,
                    meta={"cfg": cfg, "layers": layers})


def batched(count: int = 512, nmin: int = 12, nmax: int = 20, dmin: int = 4, dmax: int = 16,
            seed_cfg: int = 4) -> list:
    """cfg4: independent circuits of uneven qubit counts and depths, each with its own
    theta and TFIM field."""
    rng = np.random.default_rng(SEED_BASE + seed_cfg)
    out = []
    ns = rng.integers(nmin, nmax + 1, size=count)
    ds = rng.integers(dmin, dmax + 1, size=count)
    for b in range(count):
        n, d = int(ns[b]), int(ds[b])
        gates, P = hea_ry_rz(n, d, "cnot_ladder")
        theta = draw_theta(rng, P)
        h = float(rng.uniform(0.5, 1.5))
        out.append(Workload(name=f"batch{b}_n{n}_d{d}", n=n, gates=gates, n_params=P,
                            theta=theta, terms=tfim(n, h, periodic=False),
                            meta={"cfg": 4, "layers": d, "h": h}))
    return out


def crx_ring(n: int, layers: int) -> tuple[list, int]:
    """Controlled-rotation ansatz in the spirit of the paper's Circuit D: per layer RX(q),
    RZ(q) on every qubit, then a ring of CRX gates with their own parameters; even layers
    run q -> q+1, odd layers swap the roles of control and target and shift the ring by
    one qubit (q+1 -> q+2 read backwards)."""
    b = _Builder(n)
    for layer in range(layers):
        for q in range(n):
            b.rot("RX", q)
            b.rot("RZ", q)
        for q in range(n):
            c, t = q, (q + 1) % n
            if layer % 2:
                c, t = (q + 2) % n, (q + 1) % n
            b.ctrl("CRX", c, t)
    return b.gates, b.n_params


def random_circuit(rng: np.random.Generator, n: int, n_gates: int, share_params: bool = False,
                   kinds=("RX", "RY", "RZ", "U3", "CNOT", "CZ")) -> tuple[list, int]:
    """A random gate list over all gate kinds and qubit positions (edge-case coverage).
    With share_params, rotation gates may reuse earlier parameter indices (App. B.2)."""
    gates = []
    P = 0
    for _ in range(n_gates):
        kind = kinds[int(rng.integers(0, len(kinds)))]
        if kind in TWO_QUBIT or kind in CONTROLLED:
            if n < 2:
                continue
            a, b = (int(x) for x in rng.choice(n, size=2, replace=False))
            if kind in TWO_QUBIT:
                gates.append((kind, a, b, (-1, -1, -1)))
                continue
        else:
            a, b = int(rng.integers(0, n)), -1
        k = N_PARAMS_OF[kind]
        ps = []
        for _j in range(k):
            if share_params and P > 0 and rng.random() < 0.3:
                ps.append(int(rng.integers(0, P)))
            else:
                ps.append(P)
                P += 1
        gates.append((kind, a, b, tuple(ps) + (-1,) * (3 - k)))
    return gates, P


def random_terms(rng: np.random.Generator, n: int, count: int, wmax: int | None = None) -> list:
    return random_paulis(rng, n, count, wmax or min(4, n))
