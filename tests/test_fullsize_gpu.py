"""Parity at the workloads' full sizes, in the configuration bench.py times.

Expected values come from tests/golden/*.json, written by tests/golden/make_golden.py
with the CPU oracle only (Algorithm 1 in complex128).  At n=30 the oracle gives the
energy; the gradient there is checked by properties that hold at any size: equality
with the complex128 path and with central finite differences of the complex128 energy
on sampled parameters."""
import json
import os

import numpy as np
import pytest

from paper_2009_02823_gb300 import workloads as W
from tests.tolerances import TOL, assert_parity, energy_err, grad_err

pytestmark = pytest.mark.gpu
GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _gold(name):
    path = os.path.join(GOLD, name + ".json")
    if not os.path.exists(path):
        pytest.skip(f"fixture {name} not generated")
    with open(path) as fh:
        return json.load(fh)


def _circ(w, dtype, **kw):
    from paper_2009_02823_gb300 import Circuit
    c = Circuit(w.n, w.gates, w.n_params, dtype, **kw)
    c.set_hamiltonian(w.terms)
    return c


@pytest.mark.parametrize("dtype", ["c128", "c64"])
@pytest.mark.parametrize("cfg", [2, 5])
def test_full_gradient_vs_oracle(cfg, dtype):
    w = W.config(cfg)
    gold = _gold(f"cfg{cfg}_n{w.n}")
    assert gold["workload"] == w.name
    with _circ(w, dtype) as c:
        e, g = c.energy_and_gradient(w.theta)
    assert_parity(dtype, e, g, gold["energy"], np.array(gold["grad"]), w.name)


@pytest.mark.parametrize("spec", [2, 0])
def test_n30_bench_configuration(spec):
    """n=30, 745 gates, 200 Pauli strings, complex64 with the default fused schedule
    and checkpoints, on the specialised kernels (what bench.py times) and the generic ones."""
    w = W.config(3)
    gold = _gold(f"cfg3_n{w.n}_energy")
    with _circ(w, "c64", specialize=spec) as c:
        e64, g64 = c.energy_and_gradient(w.theta)
        assert c.plan()["checkpoints"] >= 1
        e64b, g64b = c.energy_and_gradient(w.theta)
    assert e64 == e64b and np.array_equal(g64, g64b)  # deterministic reductions
    assert energy_err(e64, gold["energy"]) <= TOL["c64"]
    if spec == 0:  # the complex128 comparison below is made once, for the benched kernels
        return
    with _circ(w, "c128") as c:
        e128, g128 = c.energy_and_gradient(w.theta)
        assert energy_err(e128, gold["energy"]) <= TOL["c128"]
        assert grad_err(g64, g128) <= TOL["c64"]
        rng = np.random.default_rng(2009)
        d = 1e-4
        for p in [0, w.n_params - 1] + list(rng.choice(w.n_params, 2, replace=False)):
            tp, tm = w.theta.copy(), w.theta.copy()
            tp[p] += d
            tm[p] -= d
            fd = (c.energy(tp) - c.energy(tm)) / (2 * d)
            assert g128[p] == pytest.approx(fd, abs=1e-7)


@pytest.mark.parametrize("dtype,arith,spec", [("c128", "fp64", 0), ("c128", "float-float", 0), ("c64", "fp64", 0),
                                              ("c64", "fp64", 2)])
def test_n29_bench_recipe_vs_oracle(dtype, arith, spec):
    """The bench recipe at n=29 (the largest size whose full Algorithm 1 gradient the
    oracle computes on a 62 GB host) against the oracle's complete gradient: the default
    fused schedule (13-qubit tiles for complex64, 12 for complex128) leaves at least 16
    fixed high index bits, as at n=30, and
    byte offsets beyond 2^32 (4 GiB per complex64 state, 8 GiB per complex128 state)."""
    w = W.config(3, n=29)
    gold = _gold(f"cfg3_n{w.n}")
    assert gold["workload"] == w.name and len(gold["grad"]) == w.n_params
    with _circ(w, dtype, c128_arith=arith, specialize=spec) as c:
        e, g = c.energy_and_gradient(w.theta)
        plan = c.plan()
    assert plan["specialized"] == spec
    assert plan["tile_qubits"] == (13 if dtype == "c64" else 12) and w.n - plan["tile_qubits"] >= 16
    if dtype == "c64":
        assert plan["checkpoints"] >= 1
    assert_parity(dtype, e, g, gold["energy"], np.array(gold["grad"]), f"{w.name} {dtype} {arith} spec={spec}")


def _central_differences(w, g64, g_gold, count=8, d=1e-4):
    """Eq. 2's derivative by central differences of the complex128 energy (FP64, step d)
    at `count` seeded parameters: truncation O(d^2) ~ 1e-9 here, against the complex64
    autograd gradient (norm-wise 1e-4) and the oracle's gradient."""
    rng = np.random.default_rng(2009_02823 + 55)
    scale = float(np.max(np.abs(g_gold)))
    with _circ(w, "c128") as c:
        for p in rng.choice(w.n_params, count, replace=False):
            tp, tm = w.theta.copy(), w.theta.copy()
            tp[p] += d
            tm[p] -= d
            fd = (c.energy(tp) - c.energy(tm)) / (2 * d)
            assert abs(g64[p] - fd) <= TOL["c64"] * scale, (p, g64[p], fd)
            assert abs(g_gold[p] - fd) <= 1e-7, (p, g_gold[p], fd)


def test_cfg5_adam_full_size():
    """n=26 U3 + CZ brickwork with TFIM: 50 Adam steps (lr 0.01) through autograd; the
    step-0 gradient equals the oracle's."""
    import torch

    from paper_2009_02823_gb300.autograd import VariationalEnergy
    w = W.config(5)
    gold = _gold(f"cfg5_n{w.n}")
    m = VariationalEnergy(w.n, w.gates, w.n_params, w.terms, "c64", theta0=w.theta, device="cuda")
    opt = torch.optim.Adam(m.parameters(), lr=0.01)
    energies = []
    for step in range(50):
        opt.zero_grad()
        e = m()
        e.backward()
        if step == 0:
            g0 = m.theta.grad.cpu().numpy()
            assert grad_err(g0, np.array(gold["grad"])) <= TOL["c64"]
            _central_differences(w, g0, np.array(gold["grad"]))
        opt.step()
        energies.append(float(e))
    assert np.all(np.isfinite(energies)) and energies[-1] < energies[0]


@pytest.mark.parametrize("n,dtype", [(33, "c64"), (31, "c128")])
def test_largest_states_closed_form(n, dtype):
    """The largest states the 280 GB device holds with room to spare (64 GiB per state at
    33 qubits complex64, 32 GiB at 31 qubits complex128): an RY layer under Hadamard^{(x)n}
    against the closed form E = prod_q f(t_q), f = (sin t + cos t)/sqrt2, and every gradient
    entry f'(t_q) prod_{r != q} f(t_r)."""
    from paper_2009_02823_gb300 import Circuit
    from tests.tolerances import assert_parity
    rng = np.random.default_rng(n)
    t = np.pi / 4 + 0.15 * rng.normal(size=n)
    gates = [("RY", q, -1, (q, -1, -1)) for q in range(n)]
    f = (np.sin(t) + np.cos(t)) / np.sqrt(2)
    df = (np.cos(t) - np.sin(t)) / np.sqrt(2)
    e_ref = float(np.prod(f))
    g_ref = np.array([df[q] * np.prod(np.delete(f, q)) for q in range(n)])
    had = np.array([[1, 1], [1, -1]]) / np.sqrt(2)
    with Circuit(n, gates, n, dtype, max_checkpoint_mib=1) as c:
        c.set_product_operator([(1.0, [had] * n)])
        e, g = c.energy_and_gradient(t)
        assert_parity(dtype, e, g, e_ref, g_ref, f"n={n}")


def _c64_vs_c128(make, tol=1e-4):
    """Run a full-size evaluation in both precisions (the complex128 path matches the
    oracle to 1e-10 at sizes the oracle finishes) and compare norm-wise."""
    out = {}
    for dtype in ("c64", "c128"):
        out[dtype] = make(dtype)
    (e64, g64), (e128, g128) = out["c64"], out["c128"]
    scale = max(float(np.max(np.abs(g128))), 1e-300)
    assert abs(e64 - e128) <= tol * max(1.0, abs(e128))
    assert float(np.max(np.abs(g64 - g128))) / scale <= tol


def test_controlled_ring_n26_precisions_agree():
    """The controlled-rotation ring (CRX on every neighbouring pair, 4 layers) at 26
    qubits: complex64 against complex128."""
    from paper_2009_02823_gb300 import Circuit
    gates, P = W.crx_ring(26, 4)
    rng = np.random.default_rng(26)
    theta = rng.uniform(0, 2 * np.pi, P)
    terms = W.random_paulis(rng, 26, 40, 4)

    def make(dtype):
        with Circuit(26, gates, P, dtype) as c:
            c.set_hamiltonian(terms)
            return c.energy_and_gradient(theta)
    _c64_vs_c128(make)


def test_non_hermitian_n26_precisions_agree():
    """A complex-coefficient operator on the 26-qubit brickwork circuit: complex64 against
    complex128 (complex expectation and gradient)."""
    from paper_2009_02823_gb300 import Circuit
    w = W.config(3, n=26, layers=4)
    rng = np.random.default_rng(27)
    terms = [(complex(c, float(rng.normal())), ops) for c, ops in w.terms]

    def make(dtype):
        with Circuit(w.n, w.gates, w.n_params, dtype) as c:
            c.set_operator(terms)
            return c.expectation_and_gradient(w.theta)
    _c64_vs_c128(make)
