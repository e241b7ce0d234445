"""complex128 in float-float arithmetic (options.c128_arith = VQG_C128_FLOAT_FLOAT) against
the CPU oracle at the complex128 bar (1e-10 relative): random circuits over every gate
kind, each compiled tile size, checkpoint restarts, non-Hermitian and tensor-product
operators with an input state, the autotuner, and the full-size golden fixtures."""
import json
import os

import numpy as np
import pytest

import oracle
from paper_2009_02823_gb300 import workloads as W
from tests.tolerances import TOL, assert_parity, energy_err

pytestmark = pytest.mark.gpu
FF = dict(c128_arith="float-float")
ALL_KINDS = ("RX", "RY", "RZ", "U3", "CNOT", "CZ", "CRX", "CRY", "CRZ", "PHASE", "CPHASE")
HAD = np.array([[1, 1], [1, -1]], dtype=complex) / np.sqrt(2)
GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _circ(n, gates, P, terms, **kw):
    from paper_2009_02823_gb300 import Circuit
    c = Circuit(n, gates, P, "c128", **FF, **kw)
    c.set_hamiltonian(terms)
    return c


@pytest.mark.parametrize("seed", range(8))
def test_random_circuits(seed):
    rng = np.random.default_rng(5000 + seed)
    n = [10, 11, 12, 13, 14, 15, 16, 13][seed]
    gates, P = W.random_circuit(rng, n, 60 + 6 * n, share_params=(seed % 3 == 0), kinds=ALL_KINDS)
    theta = rng.uniform(0, 2 * np.pi, P)
    terms = W.random_paulis(rng, n, 15, min(4, n))
    if seed == 7:
        terms.append((0.75, ()))
    e_ref, g_ref = oracle.gradient_alg1(n, gates, theta, P, terms)
    with _circ(n, gates, P, terms) as c:
        assert c.plan()["tile_qubits"] >= 10
        e, g = c.energy_and_gradient(theta)
        assert_parity("c128", e, g, e_ref, g_ref, f"float-float n={n}")
        assert energy_err(c.energy(theta), e_ref) <= TOL["c128"]
        assert np.max(np.abs(c.get_state() - oracle.state(n, gates, theta))) <= 1e-12


@pytest.mark.parametrize("K", [10, 11, 12])
@pytest.mark.parametrize("case", ["cfg2", "cfg3", "cfg5"])
def test_tile_sizes(case, K):
    n = 15
    w = W.config(int(case[3]), n=n, layers=3)
    e_ref, g_ref = oracle.gradient_alg1(n, w.gates, w.theta, w.n_params, w.terms)
    with _circ(n, w.gates, w.n_params, w.terms, tile_qubits=K) as c:
        info = c.plan()
        assert (info["tile_qubits"], info["fwd_reg_qubits"], info["rev_reg_qubits"]) == (K, 3, 3)
        e, g = c.energy_and_gradient(w.theta)
        assert_parity("c128", e, g, e_ref, g_ref, f"{case} K={K}")


@pytest.mark.parametrize("interval", [1, 3])
def test_checkpoint_restarts(interval):
    w = W.config(3, n=13, layers=4)
    e_ref, g_ref = oracle.gradient_alg1(w.n, w.gates, w.theta, w.n_params, w.terms)
    with _circ(w.n, w.gates, w.n_params, w.terms, checkpoint_interval=interval, tile_qubits=10) as c:
        assert c.plan()["checkpoints"] >= 1
        e, g = c.energy_and_gradient(w.theta)
        assert_parity("c128", e, g, e_ref, g_ref, f"ckpt={interval}")


def test_non_hermitian_operator():
    from paper_2009_02823_gb300 import Circuit
    rng = np.random.default_rng(5100)
    n = 12
    gates, P = W.random_circuit(rng, n, 90, share_params=True, kinds=ALL_KINDS)
    theta = rng.uniform(0, 2 * np.pi, P)
    terms = [(complex(c, float(rng.normal())), ops) for c, ops in W.random_paulis(rng, n, 10, 4)]
    e_ref, g_ref = oracle.gradient_alg1_operator(n, gates, theta, P, terms)
    with Circuit(n, gates, P, "c128", **FF) as c:
        c.set_operator(terms)
        e, g = c.expectation_and_gradient(theta)
    scale = float(np.max(np.abs(g_ref)))
    assert abs(e - e_ref) <= TOL["c128"] * max(1.0, abs(e_ref))
    assert float(np.max(np.abs(g - g_ref))) / scale <= TOL["c128"]


def test_products_and_input_state():
    from paper_2009_02823_gb300 import Circuit
    rng = np.random.default_rng(5200)
    n = 12
    gates, P = W.random_circuit(rng, n, 70, share_params=False, kinds=ALL_KINDS)
    theta = rng.uniform(0, 2 * np.pi, P)
    a = rng.normal(size=(2, 2)) + 1j * rng.normal(size=(2, 2))
    herm = (a + a.conj().T) / 2
    products = [(1.0, [HAD] * n), (0.4, [herm] * n)]
    psi0 = rng.normal(size=1 << n) + 1j * rng.normal(size=1 << n)
    psi0 /= np.linalg.norm(psi0)
    e_ref, g_ref = oracle.gradient_general("alg1", n, gates, theta, P, products=products, in_state=psi0)
    with Circuit(n, gates, P, "c128", **FF) as c:
        c.set_product_operator(products)
        c.set_input_state(psi0)
        e, g = c.energy_and_gradient(theta)
        assert_parity("c128", e, g, e_ref, g_ref, "products + input")


def test_autotune():
    w = W.config(3, n=16, layers=3)
    e_ref, g_ref = oracle.gradient_alg1(w.n, w.gates, w.theta, w.n_params, w.terms)
    with _circ(w.n, w.gates, w.n_params, w.terms) as c:
        r = c.autotune(w.theta)
        assert r["candidates"] >= 1 and (r["fwd_reg_qubits"], r["rev_reg_qubits"]) == (3, 3)
        e, g = c.energy_and_gradient(w.theta)
        assert_parity("c128", e, g, e_ref, g_ref, "after autotune")


@pytest.mark.parametrize("cfg", [2, 5])
def test_full_size_golden(cfg):
    """The full-size workloads (n=24 XXZ ladder, n=26 U3 brickwork) against the oracle's
    stored complex128 gradient."""
    w = W.config(cfg)
    path = os.path.join(GOLD, f"cfg{cfg}_n{w.n}.json")
    if not os.path.exists(path):
        pytest.skip("fixture not generated")
    with open(path) as fh:
        gold = json.load(fh)
    with _circ(w.n, w.gates, w.n_params, w.terms) as c:
        e, g = c.energy_and_gradient(w.theta)
    assert_parity("c128", e, g, gold["energy"], np.asarray(gold["grad"]), f"cfg{cfg} n={w.n}")


def test_n30_matches_fp64_path():
    """At the n=30 workload (745 gates, 600 parameters), float-float and FP64 complex128
    agree to the complex128 bar."""
    w = W.config(3)
    out = {}
    for arith in ("float-float", "fp64"):
        from paper_2009_02823_gb300 import Circuit
        with Circuit(w.n, w.gates, w.n_params, "c128", c128_arith=arith) as c:
            c.set_hamiltonian(w.terms)
            out[arith] = c.energy_and_gradient(w.theta)
    (e1, g1), (e2, g2) = out["float-float"], out["fp64"]
    assert_parity("c128", e1, g1, e2, g2, "n=30 float-float vs fp64")
