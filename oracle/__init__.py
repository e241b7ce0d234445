"""CPU oracle -- TEST INFRASTRUCTURE ONLY.

Only tests/, ``__graft_entry__.smoke()`` and bench.py's CPU-baseline leg may import
this package.  The product path (the CUDA library and its Python binding) never
imports, links or executes anything here, and this package never imports the
product path.  Its inputs come from the neutral workload descriptions (gate tuples
and Pauli terms as letters); it converts them with its own code below.

The arithmetic lives in ``oracle.c`` (plain C, complex128, one gate at a time); see
the header of that file for what each routine follows in the paper
(Sec. 2.2 problem statement, Algorithm 1, Algorithm 2, App. A derivatives, App. B.1
multi-parameter gates, App. B.2 repeated parameters).

Parity status: every routine is pinned by ``tests/test_oracle_pins.py`` (closed
forms, dense Kronecker brute force built from scipy's matrix exponential, Bloch-vector
products, invariants of the recurrence, finite differences).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

KIND = {"RX": 0, "RY": 1, "RZ": 2, "U3": 3, "CNOT": 4, "CZ": 5,
        "CRX": 6, "CRY": 7, "CRZ": 8, "PHASE": 9, "CPHASE": 10}
LETTER = {"I": 0, "X": 1, "Y": 2, "Z": 3}


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so (gcc, OpenMP if available)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    base = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-D_GNU_SOURCE", _SRC, "-o", _LIB + ".tmp", "-lm"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    os.replace(_LIB + ".tmp", _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        d, i, p = ctypes.c_double, ctypes.c_int, ctypes.c_void_p
        sig = {
            "oracle_gate_matrix": (None, [i, p, p]),
            "oracle_gate_derivative": (None, [i, i, p, p]),
            "oracle_apply_matrix_1q": (None, [i, p, i, p]),
            "oracle_apply_controlled_1q": (None, [i, p, i, i, p]),
            "oracle_apply_projected_1q": (None, [i, p, i, i, p]),
            "oracle_apply_gate": (None, [i, p, p, p, i]),
            "oracle_apply_gates": (None, [i, p, p, i, i, p]),
            "oracle_prepare_state": (None, [i, p, i, p, p]),
            "oracle_apply_hamiltonian": (None, [i, i, p, p, p, p]),
            "oracle_expectation": (d, [i, i, p, p, p]),
            "oracle_energy": (d, [i, p, i, p, i, p, p]),
            "oracle_gradient_parameter_shift": (None, [i, p, i, p, i, i, p, p, p, i, i]),
            "oracle_gradient_alg2": (None, [i, p, i, p, i, i, p, p, p]),
            "oracle_gradient_alg1": (None, [i, p, i, p, i, i, p, p, p, p]),
            "oracle_inner_parts": (None, [i, p, p, p]),
            "oracle_openmp_threads": (i, []),
            "oracle_apply_operator": (None, [i, i, p, p, p, p, p]),
            "oracle_apply_product_operator": (None, [i, i, p, p, p, p]),
            "oracle_gradient_ex": (None, [i, i, p, i, p, i, i, i, p, p, p, p, p, p]),
            "oracle_gradient_alg1_operator": (None, [i, p, i, p, i, i, p, p, p, p, p]),
        }
        for name, (res, args) in sig.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _lib = lib
        return lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def gate_table(gates) -> np.ndarray:
    """Neutral gate tuples -> int32 [G, 6] records (kind, q0, q1, p0, p1, p2)."""
    t = np.zeros((max(len(gates), 1), 6), dtype=np.int32)
    for i, (kind, q0, q1, ps) in enumerate(gates):
        t[i] = (KIND[kind], q0, q1, ps[0], ps[1], ps[2])
    return np.ascontiguousarray(t)


def letter_table(terms, n: int) -> tuple[np.ndarray, np.ndarray]:
    """Neutral Pauli terms -> (coef[T], letters[T, n]) with 0=I, 1=X, 2=Y, 3=Z."""
    coef = np.zeros(max(len(terms), 1), dtype=np.float64)
    let = np.zeros((max(len(terms), 1), n), dtype=np.uint8)
    for t, (c, ops) in enumerate(terms):
        coef[t] = c
        for q, l in ops:
            if let[t, q] != 0:
                raise ValueError("qubit repeated inside one Pauli string")
            let[t, q] = LETTER[l]
    return coef, np.ascontiguousarray(let)


def threads() -> int:
    return int(_load().oracle_openmp_threads())


def gate_matrix(kind: str, angles) -> np.ndarray:
    a = np.zeros(3)
    a[: len(angles)] = angles
    m = np.zeros(4, dtype=np.complex128)
    _load().oracle_gate_matrix(KIND[kind], _ptr(a), _ptr(m))
    return m.reshape(2, 2)


def gate_derivative(kind: str, slot: int, angles) -> np.ndarray:
    a = np.zeros(3)
    a[: len(angles)] = angles
    m = np.zeros(4, dtype=np.complex128)
    _load().oracle_gate_derivative(KIND[kind], slot, _ptr(a), _ptr(m))
    return m.reshape(2, 2)


def apply_matrix_1q(psi: np.ndarray, q: int, m) -> np.ndarray:
    out = np.ascontiguousarray(psi, dtype=np.complex128).copy()
    n = int(np.log2(out.size))
    mm = np.ascontiguousarray(np.asarray(m, dtype=np.complex128).reshape(4))
    _load().oracle_apply_matrix_1q(n, _ptr(out), q, _ptr(mm))
    return out


def state(n: int, gates, theta) -> np.ndarray:
    """|psi(theta)> = U_G ... U_1 |0...0>."""
    psi = np.zeros(1 << n, dtype=np.complex128)
    gt = gate_table(gates)
    th = np.ascontiguousarray(theta, dtype=np.float64)
    if th.size == 0:
        th = np.zeros(1)
    _load().oracle_prepare_state(n, _ptr(gt), len(gates), _ptr(th), _ptr(psi))
    return psi


def apply_gates(psi: np.ndarray, gates, theta, first: int = 0, last: int | None = None) -> np.ndarray:
    out = np.ascontiguousarray(psi, dtype=np.complex128).copy()
    n = int(np.log2(out.size))
    gt = gate_table(gates)
    th = np.ascontiguousarray(theta, dtype=np.float64)
    if th.size == 0:
        th = np.zeros(1)
    _load().oracle_apply_gates(n, _ptr(out), _ptr(gt), first, len(gates) if last is None else last, _ptr(th))
    return out


def apply_gate(psi: np.ndarray, gate, theta, dagger: bool = False) -> np.ndarray:
    out = np.ascontiguousarray(psi, dtype=np.complex128).copy()
    n = int(np.log2(out.size))
    gt = gate_table([gate])
    th = np.ascontiguousarray(theta, dtype=np.float64)
    if th.size == 0:
        th = np.zeros(1)
    _load().oracle_apply_gate(n, _ptr(out), _ptr(gt), _ptr(th), int(dagger))
    return out


def apply_hamiltonian(psi: np.ndarray, terms) -> np.ndarray:
    psi = np.ascontiguousarray(psi, dtype=np.complex128)
    n = int(np.log2(psi.size))
    coef, let = letter_table(terms, n)
    out = np.zeros_like(psi)
    _load().oracle_apply_hamiltonian(n, len(terms), _ptr(coef), _ptr(let), _ptr(psi), _ptr(out))
    return out


def expectation(psi: np.ndarray, terms) -> float:
    psi = np.ascontiguousarray(psi, dtype=np.complex128)
    n = int(np.log2(psi.size))
    coef, let = letter_table(terms, n)
    return float(_load().oracle_expectation(n, len(terms), _ptr(coef), _ptr(let), _ptr(psi)))


def inner(a: np.ndarray, b: np.ndarray) -> complex:
    a = np.ascontiguousarray(a, dtype=np.complex128)
    b = np.ascontiguousarray(b, dtype=np.complex128)
    n = int(np.log2(a.size))
    out = np.zeros(2)
    _load().oracle_inner_parts(n, _ptr(a), _ptr(b), _ptr(out))
    return complex(out[0], out[1])


def _args(n, gates, theta, terms):
    gt = gate_table(gates)
    th = np.ascontiguousarray(theta, dtype=np.float64)
    if th.size == 0:
        th = np.zeros(1)
    coef, let = letter_table(terms, n)
    return gt, th, coef, let


def energy(n: int, gates, theta, terms) -> float:
    gt, th, coef, let = _args(n, gates, theta, terms)
    return float(_load().oracle_energy(n, _ptr(gt), len(gates), _ptr(th), len(terms), _ptr(coef), _ptr(let)))


def gradient_parameter_shift(n: int, gates, theta, n_params: int, terms,
                             first_gate: int = 0, last_gate: int = -1) -> np.ndarray:
    """Faithful O(P^2) gradient, per-occurrence parameter shift (optionally only the
    occurrences in gates [first_gate, last_gate))."""
    gt, th, coef, let = _args(n, gates, theta, terms)
    g = np.zeros(max(n_params, 1))
    _load().oracle_gradient_parameter_shift(n, _ptr(gt), len(gates), _ptr(th), n_params, len(terms),
                                            _ptr(coef), _ptr(let), _ptr(g), first_gate, last_gate)
    return g[:n_params]


def gradient_alg2(n: int, gates, theta, n_params: int, terms) -> np.ndarray:
    """Algorithm 2 (reference gradient, derivative insertion), O(P^2)."""
    gt, th, coef, let = _args(n, gates, theta, terms)
    g = np.zeros(max(n_params, 1))
    _load().oracle_gradient_alg2(n, _ptr(gt), len(gates), _ptr(th), n_params, len(terms),
                                 _ptr(coef), _ptr(let), _ptr(g))
    return g[:n_params]


def gradient_alg1(n: int, gates, theta, n_params: int, terms) -> tuple[float, np.ndarray]:
    """Algorithm 1 (reverse mode) in the paper's order; returns (E, gradient)."""
    gt, th, coef, let = _args(n, gates, theta, terms)
    g = np.zeros(max(n_params, 1))
    e = np.zeros(1)
    _load().oracle_gradient_alg1(n, _ptr(gt), len(gates), _ptr(th), n_params, len(terms),
                                 _ptr(coef), _ptr(let), _ptr(g), _ptr(e))
    return float(e[0]), g[:n_params]


# ---------------------------------------------------------------- non-Hermitian operators (App. B.4)
def complex_letter_table(terms, n: int) -> tuple[np.ndarray, np.ndarray, np.ndarray]:
    """Terms with complex coefficients -> (re[T], im[T], letters[T, n])."""
    re_terms = [(complex(c).real, ops) for c, ops in terms]
    cr, let = letter_table(re_terms, n)
    ci = np.zeros_like(cr)
    for t, (c, _ops) in enumerate(terms):
        ci[t] = complex(c).imag
    return cr, ci, let


def apply_operator(psi: np.ndarray, terms) -> np.ndarray:
    psi = np.ascontiguousarray(psi, dtype=np.complex128)
    n = int(np.log2(psi.size))
    cr, ci, let = complex_letter_table(terms, n)
    out = np.zeros_like(psi)
    _load().oracle_apply_operator(n, len(terms), _ptr(cr), _ptr(ci), _ptr(let), _ptr(psi), _ptr(out))
    return out


def gradient_alg1_operator(n: int, gates, theta, n_params: int, terms) -> tuple[complex, np.ndarray]:
    """App. B.4: (E, dE/dtheta), both complex, for a non-Hermitian Pauli-sum operator."""
    gt = gate_table(gates)
    th = np.ascontiguousarray(theta, dtype=np.float64)
    if th.size == 0:
        th = np.zeros(1)
    cr, ci, let = complex_letter_table(terms, n)
    g = np.zeros(2 * max(n_params, 1))
    e = np.zeros(2)
    _load().oracle_gradient_alg1_operator(n, _ptr(gt), len(gates), _ptr(th), n_params, len(terms),
                                          _ptr(cr), _ptr(ci), _ptr(let), _ptr(g), _ptr(e))
    return complex(e[0], e[1]), (g[0::2] + 1j * g[1::2])[:n_params]


def gradient_parameter_shift_operator(n: int, gates, theta, n_params: int, terms) -> np.ndarray:
    """Faithful route for a non-Hermitian operator A = B + iC (B, C Hermitian: the real
    and imaginary coefficient parts of a Pauli sum): parameter shift of <B> and <C>."""
    re_terms = [(complex(c).real, ops) for c, ops in terms]
    im_terms = [(complex(c).imag, ops) for c, ops in terms]
    return (gradient_parameter_shift(n, gates, theta, n_params, re_terms)
            + 1j * gradient_parameter_shift(n, gates, theta, n_params, im_terms))


# ---------------------------------------------------------------- tensor-product operators, input states
def product_table(products, n: int) -> tuple[np.ndarray, np.ndarray]:
    """[(coef, [M_0, ..., M_{n-1}])] with 2x2 matrices per qubit -> (coef[K], mats[K, n, 4])."""
    coef = np.zeros(max(len(products), 1))
    mats = np.zeros((max(len(products), 1), n, 4), dtype=np.complex128)
    for k, (c, ms) in enumerate(products):
        if len(ms) != n:
            raise ValueError("one 2x2 matrix per qubit")
        coef[k] = c
        for q, m in enumerate(ms):
            mats[k, q] = np.asarray(m, dtype=np.complex128).reshape(4)
    return coef, np.ascontiguousarray(mats)


def apply_product_operator(psi: np.ndarray, products) -> np.ndarray:
    psi = np.ascontiguousarray(psi, dtype=np.complex128)
    n = int(np.log2(psi.size))
    coef, mats = product_table(products, n)
    out = np.zeros_like(psi)
    _load().oracle_apply_product_operator(n, len(products), _ptr(coef), _ptr(mats), _ptr(psi), _ptr(out))
    return out


def gradient_general(route: str, n: int, gates, theta, n_params: int, terms=None, products=None,
                     in_state=None) -> tuple[float, np.ndarray]:
    """(E, dE/dtheta) for a Pauli sum (terms) or a sum of tensor products (products), from
    the input state in_state (None: |0...0>).  route: "shift", "alg2" or "alg1"."""
    gt = gate_table(gates)
    th = np.ascontiguousarray(theta, dtype=np.float64)
    if th.size == 0:
        th = np.zeros(1)
    if products is not None:
        kind, nt = 1, len(products)
        coef, mats = product_table(products, n)
        let = np.zeros((1, n), dtype=np.uint8)
    else:
        kind, nt = 0, len(terms)
        coef, let = letter_table(terms, n)
        mats = np.zeros(4, dtype=np.complex128)
    ins = None
    if in_state is not None:
        ins = np.ascontiguousarray(in_state, dtype=np.complex128)
        if ins.size != 1 << n:
            raise ValueError("input state must have 2^n amplitudes")
    g = np.zeros(max(n_params, 1))
    e = np.zeros(1)
    r = {"shift": 0, "alg2": 1, "alg1": 2}[route]
    _load().oracle_gradient_ex(r, n, _ptr(gt), len(gates), _ptr(th), n_params, kind, nt, _ptr(coef),
                               _ptr(let), _ptr(mats), None if ins is None else _ptr(ins), _ptr(g), _ptr(e))
    return float(e[0]), g[:n_params]
