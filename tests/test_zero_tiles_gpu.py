"""Tiles that a |0...0> start leaves at zero (vqg_plan_pass): the planner's active-tile
counts against a support computed here from the gate list, and the results with and
without the skipping (an input state |0...0> given explicitly turns it off; clearing it
turns it back on, with forward passes that neither write nor read those zeros) against
each other and the CPU oracle (Algorithm 1, Sec. 2.3)."""
import numpy as np
import pytest

import oracle
from paper_2009_02823_gb300 import Circuit
from paper_2009_02823_gb300 import workloads as W
from tests.tolerances import TOL, assert_parity

pytestmark = pytest.mark.gpu

NONDIAG_TARGET = {"RX", "RY", "U3", "PHASE", "CNOT", "CRX", "CRY", "CRZ", "CPHASE"}


def _target(g):
    kind, q0, q1 = g[0], g[1], g[2]
    if kind in ("RX", "RY", "U3", "PHASE"):
        return q0
    if kind in ("CNOT", "CRX", "CRY", "CRZ", "CPHASE"):
        return q1
    return None  # RZ, CZ: diagonal


@pytest.mark.parametrize("n,K,spec", [(20, 12, 0), (22, 13, 2), (22, 13, 0)])
def test_active_tiles_follow_the_support(n, K, spec):
    w = W.config(3, n=n, layers=4)
    with Circuit(w.n, w.gates, w.n_params, "c64", tile_qubits=K, specialize=spec) as c:
        c.set_hamiltonian(w.terms)
        passes = c.plan_passes()
        seen = []
        support = set()
        for p in passes:
            outside = set(range(n)) - set(p["tile_qubits"])
            assert len(p["tile_qubits"]) == K and p["tiles"] == 2 ** (n - K)
            assert p["active_tiles"] == 2 ** len(outside & support), p
            for gi in p["gates"]:
                t = _target(w.gates[gi])
                if t is not None:
                    support.add(t)
            seen += p["gates"]
        assert sorted(seen) == list(range(len(w.gates)))  # every gate in exactly one pass
        assert passes[0]["active_tiles"] == 1 and passes[0]["from_zero"] == 1
        e, g = c.energy_and_gradient(w.theta)
        c.energy(w.theta)  # the state buffer holds reverse-sweep scratch after a gradient call
        psi = c.get_state()
        # an explicit |0...0> input: every tile computed, the same numbers
        zero = np.zeros(2 ** n, np.complex64)
        zero[0] = 1
        c.set_input_state(zero)
        assert all(p["active_tiles"] == p["tiles"] for p in c.plan_passes())
        e2, g2 = c.energy_and_gradient(w.theta)
        c.energy(w.theta)
        psi2 = c.get_state()
        # back to the |0...0> start: the skipping (and the unread zeros) come back
        c.set_input_state(None)
        assert c.plan_passes()[0]["active_tiles"] == 1
        e3, g3 = c.energy_and_gradient(w.theta)
    e_ref, g_ref = oracle.gradient_alg1(w.n, w.gates, w.theta, w.n_params, w.terms)
    assert_parity("c64", e, g, e_ref, g_ref, w.name)
    assert abs(e - e2) <= 1e-6 * max(1.0, abs(e)) and np.max(np.abs(g - g2)) <= 1e-6 * np.max(np.abs(g))
    assert np.max(np.abs(psi - psi2)) <= 1e-6
    assert e3 == e and np.array_equal(g3, g)


def test_active_tiles_complex128():
    """The same skipping on the complex128 kernels (FP64 and float-float tile arithmetic)."""
    w = W.config(3, n=18, layers=3)
    e_ref, g_ref = oracle.gradient_alg1(w.n, w.gates, w.theta, w.n_params, w.terms)
    for arith in ("fp64", "float-float"):
        with Circuit(w.n, w.gates, w.n_params, "c128", tile_qubits=10, c128_arith=arith) as c:
            c.set_hamiltonian(w.terms)
            assert c.plan_passes()[0]["active_tiles"] == 1
            e, g = c.energy_and_gradient(w.theta)
        assert_parity("c128", e, g, e_ref, g_ref, arith)
