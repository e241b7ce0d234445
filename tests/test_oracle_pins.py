"""Pins for the CPU oracle: each check reaches the expected value by a route other
than the oracle's own code, so a dropped term, a wrong sign or index, or a
transposed operand anywhere in oracle.c fails at least one of them.

Routes used:
  * closed forms for one qubit (RX/RY on |0>, Bloch vectors);
  * products of single-qubit Bloch components for unentangled states (pins the Y
    sign of the Pauli application and the RZ/U3 phase conventions);
  * dense brute force: scipy expm of the generators + Kronecker products (n <= 5);
  * invariants of the recurrence of Sec. 2.2 (the pair <lambda_i|phi_{i+1}> is
    constant and equals E; phi returns to |0...0>; norms are conserved);
  * central finite differences (Eq. 2, symmetric form; truncation O(delta^2));
  * the chain-rule sum for repeated parameters (App. B.2);
  * the variational bound E >= lowest eigenvalue of H.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2009_02823_gb300 import workloads as W
from tests import dense_ref as D

pytestmark = pytest.mark.filterwarnings("ignore")


# ---------------------------------------------------------------- closed forms
@pytest.mark.parametrize("t", [0.0, 0.3, 1.1, 2.0, math.pi, 4.4, 5.9])
def test_rx_on_zero_with_z(t):
    """RX(t)|0> under H = Z: E = cos t, dE/dt = -sin t."""
    gates = [("RX", 0, -1, (0, -1, -1))]
    terms = [(1.0, ((0, "Z"),))]
    th = np.array([t])
    assert oracle.energy(1, gates, th, terms) == pytest.approx(math.cos(t), abs=1e-14)
    for g in (oracle.gradient_parameter_shift(1, gates, th, 1, terms),
              oracle.gradient_alg2(1, gates, th, 1, terms),
              oracle.gradient_alg1(1, gates, th, 1, terms)[1]):
        assert g[0] == pytest.approx(-math.sin(t), abs=1e-14)


@pytest.mark.parametrize("t", [0.2, 1.3, 2.9, 4.1])
def test_single_qubit_bloch_components(t):
    """RX(t)|0> has Bloch vector (0, -sin t, cos t); RY(t)|0> has (sin t, 0, cos t)."""
    th = np.array([t])
    rx = [("RX", 0, -1, (0, -1, -1))]
    ry = [("RY", 0, -1, (0, -1, -1))]
    X, Y = [(1.0, ((0, "X"),))], [(1.0, ((0, "Y"),))]
    assert oracle.energy(1, rx, th, X) == pytest.approx(0.0, abs=1e-14)
    assert oracle.energy(1, rx, th, Y) == pytest.approx(-math.sin(t), abs=1e-14)
    assert oracle.energy(1, ry, th, X) == pytest.approx(math.sin(t), abs=1e-14)
    assert oracle.energy(1, ry, th, Y) == pytest.approx(0.0, abs=1e-14)
    assert oracle.gradient_alg1(1, ry, th, 1, X)[1][0] == pytest.approx(math.cos(t), abs=1e-14)
    assert oracle.gradient_alg1(1, rx, th, 1, Y)[1][0] == pytest.approx(-math.cos(t), abs=1e-14)


def _bloch_product_case(seed, n, use_u3):
    rng = np.random.default_rng(seed)
    gates, P = [], 0
    for q in range(n):
        if use_u3:
            gates.append(("U3", q, -1, (P, P + 1, P + 2)))
            P += 3
        else:
            gates.append(("RY", q, -1, (P, -1, -1)))
            gates.append(("RZ", q, -1, (P + 1, -1, -1)))
            P += 2
    theta = rng.uniform(0, 2 * np.pi, P)
    terms = W.random_paulis(rng, n, 12, min(4, n))
    return gates, P, theta, terms


def _bloch(theta, q, use_u3):
    """Polar/azimuth of qubit q: RY(t) then RZ(f) gives (sin t cos f, sin t sin f, cos t);
    U3(t, f, l)|0> = (cos t/2, e^{if} sin t/2) has the same vector, independent of l."""
    t, f = (theta[3 * q], theta[3 * q + 1]) if use_u3 else (theta[2 * q], theta[2 * q + 1])
    return np.array([math.sin(t) * math.cos(f), math.sin(t) * math.sin(f), math.cos(t)])


@pytest.mark.parametrize("use_u3", [False, True])
@pytest.mark.parametrize("seed", [1, 2, 3])
def test_unentangled_pauli_products(seed, use_u3):
    n = 5
    gates, P, theta, terms = _bloch_product_case(seed, n, use_u3)
    expect = 0.0
    for c, ops in terms:
        v = c
        for q, l in ops:
            v *= _bloch(theta, q, use_u3)["XYZ".index(l)]
        expect += v
    assert oracle.energy(n, gates, theta, terms) == pytest.approx(expect, abs=1e-13)
    # gradient of the product closed form by central differences of the closed form
    g = oracle.gradient_alg1(n, gates, theta, P, terms)[1]
    for p in range(P):
        d = 1e-6
        tp, tm = theta.copy(), theta.copy()
        tp[p] += d
        tm[p] -= d

        def f(th):
            s = 0.0
            for c, ops in terms:
                v = c
                for q, l in ops:
                    v *= _bloch(th, q, use_u3)["XYZ".index(l)]
                s += v
            return s
        assert g[p] == pytest.approx((f(tp) - f(tm)) / (2 * d), abs=1e-8)
    if use_u3:  # the lambda slot leaves the Bloch vector alone
        assert np.allclose(g[2::3], 0.0, atol=1e-13)


# ---------------------------------------------------------------- dense brute force
@pytest.mark.parametrize("kind", ["RX", "RY", "RZ", "U3"])
def test_gate_matrices_vs_expm(kind):
    rng = np.random.default_rng(7)
    for _ in range(5):
        a = rng.uniform(-7, 7, 3)
        m = oracle.gate_matrix(kind, a)
        ref = {"RX": D.rot(D.X, a[0]), "RY": D.rot(D.Y, a[0]), "RZ": D.rot(D.Z, a[0]),
               "U3": D.u3(*a)}[kind]
        assert np.allclose(m, ref, atol=1e-14)
        k = 3 if kind == "U3" else 1
        for slot in range(k):
            h = 1e-6
            ap, am = a.copy(), a.copy()
            ap[slot] += h
            am[slot] -= h
            fp = D.u3(*ap) if kind == "U3" else D.rot({"RX": D.X, "RY": D.Y, "RZ": D.Z}[kind], ap[0])
            fm = D.u3(*am) if kind == "U3" else D.rot({"RX": D.X, "RY": D.Y, "RZ": D.Z}[kind], am[0])
            assert np.allclose(oracle.gate_derivative(kind, slot, a), (fp - fm) / (2 * h), atol=1e-9)


@pytest.mark.parametrize("seed", range(6))
def test_random_circuits_vs_dense(seed):
    rng = np.random.default_rng(100 + seed)
    n = int(rng.integers(1, 6))
    kinds = ("RX", "RY", "RZ", "U3") if n == 1 else ("RX", "RY", "RZ", "U3", "CNOT", "CZ")
    gates, P = W.random_circuit(rng, n, 14, share_params=(seed % 2 == 1), kinds=kinds)
    theta = rng.uniform(0, 2 * np.pi, max(P, 1))
    terms = W.random_paulis(rng, n, 6, min(4, n))
    # state and Hamiltonian application
    psi = oracle.state(n, gates, theta)
    assert np.allclose(psi, D.state(n, gates, theta), atol=1e-13)
    assert np.allclose(oracle.apply_hamiltonian(psi, terms), D.hamiltonian(terms, n) @ psi, atol=1e-13)
    e_ref = D.energy(n, gates, theta, terms)
    assert oracle.energy(n, gates, theta, terms) == pytest.approx(e_ref, abs=1e-13)
    g_ref = D.gradient_shift(n, gates, theta, P, terms)
    g_fd = D.gradient_fd(n, gates, theta, P, terms)
    assert np.allclose(g_ref, g_fd, atol=1e-8)
    e1, g1 = oracle.gradient_alg1(n, gates, theta, P, terms)
    assert e1 == pytest.approx(e_ref, abs=1e-13)
    assert np.allclose(g1, g_ref, atol=1e-12)
    assert np.allclose(oracle.gradient_alg2(n, gates, theta, P, terms), g_ref, atol=1e-12)
    assert np.allclose(oracle.gradient_parameter_shift(n, gates, theta, P, terms), g_ref, atol=1e-12)


def test_entangler_action_on_basis_states():
    """CNOT(c->t) flips t exactly where c = 1; CZ negates exactly the |..1..1..> states."""
    n = 3
    for j in range(8):
        e = np.zeros(8, complex)
        e[j] = 1
        out = oracle.apply_gate(e, ("CNOT", 2, 0, (-1, -1, -1)), [0.0])
        k = j ^ 1 if (j >> 2) & 1 else j
        assert out[k] == 1 and abs(out).sum() == 1
        out = oracle.apply_gate(e, ("CZ", 0, 1, (-1, -1, -1)), [0.0])
        assert out[j] == (-1 if (j & 3) == 3 else 1)


def test_pauli_strings_vs_kron():
    rng = np.random.default_rng(5)
    n = 4
    psi = rng.standard_normal(16) + 1j * rng.standard_normal(16)
    for letters in ["XIII", "IYII", "IIZI", "YYYY", "XYZX", "ZZII", "IXYI"]:
        ops = tuple((q, l) for q, l in enumerate(letters) if l != "I")
        term = [(0.7, ops)]
        assert np.allclose(oracle.apply_hamiltonian(psi, term), D.hamiltonian(term, n) @ psi, atol=1e-13)


# ---------------------------------------------------------------- invariants
def test_recurrence_invariants_cfg1():
    """Along the reverse recurrence phi_i = U_i^dag phi_{i+1}, lambda_i = U_{i+1}^dag lambda_{i+1}
    (Sec. 2.2), <lambda|phi> stays equal to E, norms are conserved, and phi ends at |0...0>."""
    w = W.config(1)
    psi = oracle.state(w.n, w.gates, w.theta)
    assert np.linalg.norm(psi) == pytest.approx(1.0, abs=1e-13)
    lam = oracle.apply_hamiltonian(psi, w.terms)
    e = oracle.energy(w.n, w.gates, w.theta, w.terms)
    nl = np.linalg.norm(lam)
    phi = psi.copy()
    for i in reversed(range(w.n_gates)):
        assert oracle.inner(lam, phi).real == pytest.approx(e, abs=1e-12)
        phi = oracle.apply_gate(phi, w.gates[i], w.theta, dagger=True)
        lam = oracle.apply_gate(lam, w.gates[i], w.theta, dagger=True)
        assert np.linalg.norm(lam) == pytest.approx(nl, rel=1e-12)
    zero = np.zeros_like(phi)
    zero[0] = 1
    assert np.allclose(phi, zero, atol=1e-12)


def test_three_routes_agree_cfg1():
    w = W.config(1)
    e1, g1 = oracle.gradient_alg1(w.n, w.gates, w.theta, w.n_params, w.terms)
    g2 = oracle.gradient_alg2(w.n, w.gates, w.theta, w.n_params, w.terms)
    g3 = oracle.gradient_parameter_shift(w.n, w.gates, w.theta, w.n_params, w.terms)
    assert e1 == pytest.approx(oracle.energy(w.n, w.gates, w.theta, w.terms), abs=1e-13)
    assert np.abs(g1 - g2).max() < 1e-12
    assert np.abs(g1 - g3).max() < 1e-12


def test_central_difference_cfg1_subset():
    """Eq. 2 in symmetric form with delta = 1e-4 in FP64: truncation ~ delta^2 |E'''|/6."""
    w = W.config(1)
    g = oracle.gradient_alg1(w.n, w.gates, w.theta, w.n_params, w.terms)[1]
    rng = np.random.default_rng(11)
    for p in rng.choice(w.n_params, 10, replace=False):
        d = 1e-4
        tp, tm = w.theta.copy(), w.theta.copy()
        tp[p] += d
        tm[p] -= d
        fd = (oracle.energy(w.n, w.gates, tp, w.terms) - oracle.energy(w.n, w.gates, tm, w.terms)) / (2 * d)
        assert g[p] == pytest.approx(fd, abs=1e-7)


def test_repeated_parameters_chain_rule():
    """App. B.2: renaming every occurrence to a fresh parameter and summing the entries
    of the renamed gradient gives the gradient of the shared parametrisation."""
    rng = np.random.default_rng(21)
    n = 4
    gates, P = W.random_circuit(rng, n, 30, share_params=True)
    theta = rng.uniform(0, 2 * np.pi, P)
    terms = W.random_paulis(rng, n, 8, 3)
    fresh, fmap, k = [], [], 0
    for kind, q0, q1, ps in gates:
        nps = []
        for p in ps:
            if p < 0:
                nps.append(-1)
            else:
                nps.append(k)
                fmap.append(p)
                k += 1
        fresh.append((kind, q0, q1, tuple(nps)))
    ftheta = theta[np.array(fmap)]
    gf = oracle.gradient_alg1(n, fresh, ftheta, k, terms)[1]
    summed = np.zeros(P)
    np.add.at(summed, np.array(fmap), gf)
    g = oracle.gradient_alg1(n, gates, theta, P, terms)[1]
    assert np.allclose(g, summed, atol=1e-13)
    assert np.allclose(g, D.gradient_shift(n, gates, theta, P, terms), atol=1e-12)


def test_variational_bound():
    w = W.config(1, n=6, layers=2)
    h = D.hamiltonian(w.terms, w.n)
    e0 = np.linalg.eigvalsh(h)[0]
    rng = np.random.default_rng(3)
    for _ in range(5):
        th = rng.uniform(0, 2 * np.pi, w.n_params)
        assert oracle.energy(w.n, w.gates, th, w.terms) >= e0 - 1e-12


def test_hermitian_gradient_is_real_and_energy_matches_expectation():
    w = W.config(5, n=5, layers=2)
    psi = oracle.state(w.n, w.gates, w.theta)
    e = oracle.expectation(psi, w.terms)
    lam = oracle.apply_hamiltonian(psi, w.terms)
    assert abs(oracle.inner(psi, lam).imag) < 1e-13
    assert e == pytest.approx(oracle.energy(w.n, w.gates, w.theta, w.terms), abs=1e-14)
    g_ref = D.gradient_shift(w.n, w.gates, w.theta, w.n_params, w.terms)
    assert np.allclose(oracle.gradient_alg1(w.n, w.gates, w.theta, w.n_params, w.terms)[1], g_ref, atol=1e-12)


# ---------------------------------------------------------------- controlled and phase gates (App. A)
@pytest.mark.parametrize("t", [0.0, 0.4, 1.7, 3.0, 5.2])
def test_controlled_rx_closed_form(t):
    """CRX(t) with the control prepared in |1> (RX(pi)) acts as RX(t) on the target:
    <Z_t> = cos t, d/dt = -sin t; with the control in |0> nothing happens (E = 1, 0);
    with the control in |+> (RY(pi/2)) the two branches average: (1 + cos t)/2."""
    th = np.array([np.pi, t])
    z_t = [(1.0, ((1, "Z"),))]
    on = [("RX", 0, -1, (0, -1, -1)), ("CRX", 0, 1, (1, -1, -1))]
    plus = [("RY", 0, -1, (0, -1, -1)), ("CRX", 0, 1, (1, -1, -1))]
    off = [("CRX", 0, 1, (0, -1, -1))]
    assert oracle.energy(2, on, th, z_t) == pytest.approx(math.cos(t), abs=1e-14)
    assert oracle.energy(2, off, np.array([t]), z_t) == pytest.approx(1.0, abs=1e-14)
    thp = np.array([np.pi / 2, t])
    assert oracle.energy(2, plus, thp, z_t) == pytest.approx(0.5 * (1 + math.cos(t)), abs=1e-14)
    for route in (oracle.gradient_parameter_shift, oracle.gradient_alg2, lambda *a: oracle.gradient_alg1(*a)[1]):
        assert route(2, on, th, 2, z_t)[1] == pytest.approx(-math.sin(t), abs=1e-13)
        assert route(2, off, np.array([t]), 1, z_t)[0] == pytest.approx(0.0, abs=1e-13)
        assert route(2, plus, thp, 2, z_t)[1] == pytest.approx(-0.5 * math.sin(t), abs=1e-13)


@pytest.mark.parametrize("t", [0.3, 1.9, 4.0])
def test_phase_gate_closed_form(t):
    """PHASE(t) on |+> = RY(pi/2)|0>: Bloch vector (cos t, sin t, 0)."""
    gates = [("RY", 0, -1, (0, -1, -1)), ("PHASE", 0, -1, (1, -1, -1))]
    th = np.array([np.pi / 2, t])
    X, Y = [(1.0, ((0, "X"),))], [(1.0, ((0, "Y"),))]
    assert oracle.energy(1, gates, th, X) == pytest.approx(math.cos(t), abs=1e-14)
    assert oracle.energy(1, gates, th, Y) == pytest.approx(math.sin(t), abs=1e-14)
    for route in (oracle.gradient_parameter_shift, oracle.gradient_alg2, lambda *a: oracle.gradient_alg1(*a)[1]):
        assert route(1, gates, th, 2, X)[1] == pytest.approx(-math.sin(t), abs=1e-13)
        assert route(1, gates, th, 2, Y)[1] == pytest.approx(math.cos(t), abs=1e-13)


@pytest.mark.parametrize("kind", ["CRX", "CRY", "CRZ", "PHASE", "CPHASE"])
def test_controlled_gates_vs_expm(kind):
    """Two-qubit unitary of each new kind (control 0, target 1; PHASE on qubit 0) against
    expm of its generator on the full space, and the oracle's derivative route (App. A:
    target derivative, then the control projection) against dU/dt = -i G U."""
    rng = np.random.default_rng(3)
    gate = (kind, 0, -1 if kind == "PHASE" else 1, (0, -1, -1))
    n = 1 if kind == "PHASE" else 2
    for _ in range(4):
        t = float(rng.uniform(-7, 7))
        U = D.gate_unitary(gate, [t], n)
        cols = np.stack([oracle.apply_gate(np.eye(1 << n, dtype=complex)[:, k], gate, np.array([t]))
                         for k in range(1 << n)], axis=1)
        assert np.allclose(cols, U, atol=1e-14)
        dU = -1j * D.generator(gate, n) @ U
        # derivative route = Algorithm 2 on a one-gate circuit with H = |k><l| parts
        for k in range(1 << n):
            psi = np.eye(1 << n, dtype=complex)[:, k]
            d = oracle.gate_derivative(kind, 0, [t])
            out = oracle.apply_matrix_1q(psi, 1 if n == 2 else 0, d)
            if kind != "PHASE":
                out = np.where((np.arange(1 << n) & 1) != 0, out, 0)  # project control 0 onto 1
            assert np.allclose(out, dU[:, k], atol=1e-13)


@pytest.mark.parametrize("seed", range(6))
def test_random_controlled_circuits_vs_dense(seed):
    """Random circuits over every gate kind: state and energy against the dense route;
    the three oracle gradient routes (including the four-term shift rule of the
    controlled rotations) against the dense generator-insertion gradient and central
    differences."""
    rng = np.random.default_rng(300 + seed)
    n = int(rng.integers(2, 6))
    kinds = ("RX", "RY", "RZ", "CNOT", "CZ", "CRX", "CRY", "CRZ", "PHASE", "CPHASE")
    gates, P = W.random_circuit(rng, n, 16, share_params=(seed % 2 == 1), kinds=kinds)
    theta = rng.uniform(0, 2 * np.pi, max(P, 1))[:P]
    terms = W.random_paulis(rng, n, 6, min(4, n))
    psi = oracle.state(n, gates, theta)
    assert np.allclose(psi, D.state(n, gates, theta), atol=1e-13)
    e_ref = D.energy(n, gates, theta, terms)
    assert oracle.energy(n, gates, theta, terms) == pytest.approx(e_ref, abs=1e-13)
    g_ref = D.gradient_generator(n, gates, theta, P, terms)
    assert np.allclose(g_ref, D.gradient_fd(n, gates, theta, P, terms), atol=1e-8)
    e1, g1 = oracle.gradient_alg1(n, gates, theta, P, terms)
    assert e1 == pytest.approx(e_ref, abs=1e-13)
    assert np.allclose(g1, g_ref, atol=1e-12)
    assert np.allclose(oracle.gradient_alg2(n, gates, theta, P, terms), g_ref, atol=1e-12)
    assert np.allclose(oracle.gradient_parameter_shift(n, gates, theta, P, terms), g_ref, atol=1e-12)


def test_two_term_shift_fails_for_controlled_rotation():
    """The plain two-term rule is not exact for a controlled rotation (frequencies 1/2
    and 1): a check that the four-term rule is needed, not an accident of the data."""
    gates = [("U3", 0, -1, (0, 1, 2)), ("U3", 1, -1, (3, 4, 5)), ("CRY", 0, 1, (6, -1, -1))]
    th = np.array([0.7, 0.4, 1.1, 1.3, 0.2, 2.1, 0.9])
    terms = [(1.0, ((1, "X"),)), (0.6, ((1, "Z"),)), (0.3, ((0, "Y"), (1, "X")))]
    g_ref = D.gradient_fd(2, gates, th, 7, terms)
    two = 0.5 * (D.energy(2, gates, th, terms, (2, 0, np.pi / 2)) - D.energy(2, gates, th, terms, (2, 0, -np.pi / 2)))
    assert abs(two - g_ref[6]) > 1e-3
    assert oracle.gradient_parameter_shift(2, gates, th, 7, terms)[6] == pytest.approx(g_ref[6], abs=1e-9)


# ---------------------------------------------------------------- non-Hermitian operators (App. B.4)
@pytest.mark.parametrize("t", [0.0, 0.5, 2.2, 4.9])
def test_non_hermitian_closed_form(t):
    """RY(t)|0> under A = Z + iX: <A> = cos t + i sin t = e^{it}, dA/dt = i e^{it}.
    RX(t)|0> under A = X + iY: <A> = -i sin t, d/dt = -i cos t."""
    ry = [("RY", 0, -1, (0, -1, -1))]
    rx = [("RX", 0, -1, (0, -1, -1))]
    th = np.array([t])
    a1 = [(1.0, ((0, "Z"),)), (1j, ((0, "X"),))]
    a2 = [(1.0, ((0, "X"),)), (1j, ((0, "Y"),))]
    e, g = oracle.gradient_alg1_operator(1, ry, th, 1, a1)
    assert e == pytest.approx(np.exp(1j * t), abs=1e-14)
    assert g[0] == pytest.approx(1j * np.exp(1j * t), abs=1e-14)
    e, g = oracle.gradient_alg1_operator(1, rx, th, 1, a2)
    assert e == pytest.approx(-1j * math.sin(t), abs=1e-14)
    assert g[0] == pytest.approx(-1j * math.cos(t), abs=1e-14)
    for terms, gates in ((a1, ry), (a2, rx)):
        ps = oracle.gradient_parameter_shift_operator(1, gates, th, 1, terms)
        assert ps[0] == pytest.approx(oracle.gradient_alg1_operator(1, gates, th, 1, terms)[1][0], abs=1e-14)


@pytest.mark.parametrize("seed", range(5))
def test_non_hermitian_vs_dense(seed):
    """Random circuits and complex-coefficient Pauli sums: the operator application, the
    complex expectation and the App. B.4 gradient against the dense route (Kronecker
    products, central differences of the complex expectation); the parameter-shift
    route on the real and imaginary parts agrees too."""
    rng = np.random.default_rng(700 + seed)
    n = int(rng.integers(1, 6))
    kinds = ("RX", "RY", "RZ", "U3") if n == 1 else ("RX", "RY", "RZ", "U3", "CNOT", "CZ", "CRX", "PHASE")
    gates, P = W.random_circuit(rng, n, 12, share_params=(seed % 2 == 0), kinds=kinds)
    theta = rng.uniform(0, 2 * np.pi, max(P, 1))[:P]
    terms = [(complex(c, float(rng.normal())), ops) for c, ops in W.random_paulis(rng, n, 6, min(4, n))]
    psi = oracle.state(n, gates, theta)
    assert np.allclose(oracle.apply_operator(psi, terms), D.operator(terms, n) @ psi, atol=1e-13)
    e_ref = D.expectation_complex(n, gates, theta, terms)
    g_ref = D.gradient_fd_complex(n, gates, theta, P, terms)
    e, g = oracle.gradient_alg1_operator(n, gates, theta, P, terms)
    assert e == pytest.approx(e_ref, abs=1e-13)
    assert np.allclose(g, g_ref, atol=1e-8)
    assert np.allclose(oracle.gradient_parameter_shift_operator(n, gates, theta, P, terms), g, atol=1e-12)


def test_non_hermitian_reduces_to_hermitian():
    """Real coefficients: the App. B.4 route returns the Algorithm-1 energy and gradient
    with zero imaginary parts."""
    w = W.config(1, n=6, layers=2)
    e, g = oracle.gradient_alg1_operator(w.n, w.gates, w.theta, w.n_params, w.terms)
    e1, g1 = oracle.gradient_alg1(w.n, w.gates, w.theta, w.n_params, w.terms)
    assert e.real == pytest.approx(e1, abs=1e-13) and abs(e.imag) < 1e-13
    assert np.allclose(g.real, g1, atol=1e-13) and np.allclose(g.imag, 0.0, atol=1e-13)


# ---------------------------------------------------------------- tensor-product operators and input states
HAD = np.array([[1, 1], [1, -1]], dtype=complex) / np.sqrt(2)


@pytest.mark.parametrize("n", [1, 3, 5])
def test_hadamard_product_closed_form(n):
    """The paper's benchmark operator H^{(x)N} (Sec. 3) on an unentangled RY layer:
    <H> per qubit is (sin t + cos t)/sqrt2, so E = prod_q f(t_q) and
    dE/dt_q = f'(t_q) prod_{r != q} f(t_r), for all three routes."""
    rng = np.random.default_rng(n)
    t = rng.uniform(0, 2 * np.pi, n)
    gates = [("RY", q, -1, (q, -1, -1)) for q in range(n)]
    f = (np.sin(t) + np.cos(t)) / np.sqrt(2)
    df = (np.cos(t) - np.sin(t)) / np.sqrt(2)
    e_ref = float(np.prod(f))
    g_ref = np.array([df[q] * np.prod(np.delete(f, q)) for q in range(n)])
    for route in ("shift", "alg2", "alg1"):
        e, g = oracle.gradient_general(route, n, gates, t, n, products=[(1.0, [HAD] * n)])
        assert e == pytest.approx(e_ref, abs=1e-13)
        assert np.allclose(g, g_ref, atol=1e-13)


def _random_hermitian(rng):
    a = rng.normal(size=(2, 2)) + 1j * rng.normal(size=(2, 2))
    return (a + a.conj().T) / 2


@pytest.mark.parametrize("seed", range(5))
def test_products_and_input_state_vs_dense(seed):
    """Sums of tensor products of random Hermitian 2x2 matrices and a random input state:
    the operator application, the energy and the three gradient routes against the dense
    route (Kronecker products, central differences)."""
    rng = np.random.default_rng(800 + seed)
    n = int(rng.integers(1, 6))
    kinds = ("RX", "RY", "RZ", "U3") if n == 1 else ("RX", "RY", "RZ", "U3", "CNOT", "CZ", "CRY", "PHASE")
    gates, P = W.random_circuit(rng, n, 12, share_params=(seed % 2 == 0), kinds=kinds)
    theta = rng.uniform(0, 2 * np.pi, max(P, 1))[:P]
    products = [(float(rng.normal()), [_random_hermitian(rng) for _ in range(n)]) for _ in range(1 + seed % 3)]
    psi0 = rng.normal(size=1 << n) + 1j * rng.normal(size=1 << n)
    if seed % 2:
        psi0 /= np.linalg.norm(psi0)  # normalised or not: E is the plain quadratic form
    A = np.zeros((1 << n, 1 << n), dtype=complex)
    for c, ms in products:
        A += c * D.lift(dict(enumerate(ms)), n)
    assert np.allclose(oracle.apply_product_operator(psi0, products), A @ psi0, atol=1e-13)

    def dense_e(th):
        psi = psi0.copy()
        for g in gates:
            psi = D.gate_unitary(g, th, n) @ psi
        return float(np.real(psi.conj() @ A @ psi))

    e_ref = dense_e(theta)
    g_ref = np.zeros(P)
    for p in range(P):
        tp, tm = theta.copy(), theta.copy()
        tp[p] += 1e-5
        tm[p] -= 1e-5
        g_ref[p] = (dense_e(tp) - dense_e(tm)) / 2e-5
    for route in ("shift", "alg2", "alg1"):
        e, g = oracle.gradient_general(route, n, gates, theta, P, products=products, in_state=psi0)
        assert e == pytest.approx(e_ref, abs=1e-12)
        assert np.allclose(g, g_ref, atol=1e-7 * max(1.0, np.max(np.abs(g_ref))))
    # Pauli operator from a custom input state too
    terms = W.random_paulis(rng, n, 5, min(4, n))
    Hm = D.hamiltonian(terms, n)
    psi = psi0.copy()
    for g in gates:
        psi = D.gate_unitary(g, theta, n) @ psi
    e, _g = oracle.gradient_general("alg1", n, gates, theta, P, terms=terms, in_state=psi0)
    assert e == pytest.approx(float(np.real(psi.conj() @ Hm @ psi)), abs=1e-12)
