"""Per-pass specialised kernels (options.specialize): the complex64 tile passes run kernels
generated for the circuit's own passes.  On the host the generated sources must compile
(vqg_specialize_prepare); on the GPU the results must match the CPU oracle (Algorithm 1,
Sec. 2.3) at the complex64 bar and the generic kernels' results."""
import numpy as np
import pytest

from paper_2009_02823_gb300 import binding as B
from paper_2009_02823_gb300 import workloads as W
from tests.tolerances import TOL, assert_parity


def test_prepare_compiles_on_host(tmp_path, monkeypatch):
    monkeypatch.setenv("VQG_SPEC_CACHE", str(tmp_path))
    w = W.config(3, n=11, layers=2)
    nk = B.specialize_prepare(w.n, w.gates, w.n_params)
    assert nk >= 1
    assert len(list(tmp_path.glob("*.cubin"))) == nk
    assert B.specialize_prepare(w.n, w.gates, w.n_params) == nk  # served from the cache
    # below the fused size there is nothing to compile
    w8 = W.config(1, n=8, layers=1)
    assert B.specialize_prepare(w8.n, w8.gates, w8.n_params) == 0


def _cases():
    rng = np.random.default_rng(2024)
    out = []
    for n, kinds in ((12, ("RX", "RY", "RZ", "U3", "CNOT", "CZ")),
                     (13, ("RX", "RY", "RZ", "CNOT", "CZ", "CRX", "CRY", "CRZ", "PHASE", "CPHASE"))):
        gates, P = W.random_circuit(rng, n, 90, share_params=True, kinds=kinds)
        out.append((f"random{n}", n, gates, P, rng.uniform(0, 2 * np.pi, P), W.random_paulis(rng, n, 12, 4)))
    w = W.config(3, n=14, layers=4)
    out.append((w.name, w.n, w.gates, w.n_params, w.theta, w.terms))
    w = W.config(5, n=12, layers=3)
    out.append((w.name, w.n, w.gates, w.n_params, w.theta, w.terms))
    return out


@pytest.mark.gpu
@pytest.mark.parametrize("case", _cases(), ids=lambda c: c[0])
def test_specialized_matches_oracle_and_generic(case):
    import oracle
    name, n, gates, P, theta, terms = case
    e_ref, g_ref = oracle.gradient_alg1(n, gates, theta, P, terms)
    with B.Circuit(n, gates, P, "c64") as c:
        c.set_hamiltonian(terms)
        e0, g0 = c.energy_and_gradient(theta)
    for level, ck in ((1, 0), (2, 0), (2, -1)):  # checkpoints at every pass boundary, and none
        with B.Circuit(n, gates, P, "c64", specialize=level, checkpoint_interval=ck) as c:
            c.set_hamiltonian(terms)
            assert c.plan()["specialized"] == level
            e, g = c.energy_and_gradient(theta)
            assert_parity("c64", e, g, e_ref, g_ref, name)
            assert abs(c.energy(theta) - e_ref) <= TOL["c64"] * max(1.0, abs(e_ref))
            psi = c.get_state()
            assert np.max(np.abs(psi - oracle.state(n, gates, theta))) <= 2e-5
    # same arithmetic as the generic kernels
    assert abs(e - e0) <= 1e-6 * max(1.0, abs(e0))
    assert np.max(np.abs(g - g0)) <= 1e-6 * max(1.0, np.max(np.abs(g0)))


@pytest.mark.gpu
def test_specialized_diagnostics_and_graph():
    w = W.config(3, n=13, layers=5)
    with B.Circuit(w.n, w.gates, w.n_params, "c64", specialize=2, use_graph=True) as c:
        c.set_hamiltonian(w.terms)
        r1 = c.energy_and_gradient(w.theta)
        r2 = c.energy_and_gradient(w.theta)  # replayed from the captured graph
        assert r1[0] == r2[0] and np.array_equal(r1[1], r2[1])
        c.set_diagnostics(True)
        c.energy_and_gradient(w.theta)
        d = c.diagnostics()
    assert d["checkpoints"] >= 1
    for x in d["entries"]:
        assert abs(x["lam_phi_re"] - d["energy"]) <= 1e-4 * max(1.0, abs(d["energy"]))


@pytest.mark.gpu
def test_specialized_hamiltonian_edge_cases():
    """No diagonal terms (the x = 0 group is empty), a group mixing real and imaginary
    weights, and a non-Hermitian operator (its two Hermitian parts swap Hamiltonian tables
    between the runs), through the specialised kernels."""
    import oracle
    n = 12
    rng = np.random.default_rng(8)
    gates, P = W.random_circuit(rng, n, 70, share_params=False)
    theta = rng.uniform(0, 2 * np.pi, P)
    terms = [(c, ops) for c, ops in W.random_paulis(rng, n, 14, 4) if any(l in "XY" for _q, l in ops)]
    terms += [(-0.23, ((3, "X"),)), (1.31, ((3, "Y"),)), (0.4, ((1, "Y"), (5, "Y")))]
    e_ref, g_ref = oracle.gradient_alg1(n, gates, theta, P, terms)
    with B.Circuit(n, gates, P, "c64", specialize=1) as c:
        c.set_hamiltonian(terms)
        e, g = c.energy_and_gradient(theta)
        assert_parity("c64", e, g, e_ref, g_ref, "no diagonal terms")
        cterms = [(complex(cf, 0.5 * cf), ops) for cf, ops in W.random_paulis(rng, n, 10, 3)]
        c.set_operator(cterms)
        ex, gx = c.expectation_and_gradient(theta)
    ex_ref, gx_ref = oracle.gradient_alg1_operator(n, gates, theta, P, cterms)
    assert abs(ex - ex_ref) <= TOL["c64"] * max(1.0, abs(ex_ref))
    assert np.max(np.abs(gx - gx_ref)) <= TOL["c64"] * max(1e-300, np.max(np.abs(gx_ref)))


@pytest.mark.gpu
@pytest.mark.parametrize("n,layers", [(16, 4), (17, 3)])
def test_specialized_13_qubit_tiles(n, layers):
    """The bench recipe with 13-qubit tiles at sizes the oracle finishes quickly: several
    passes, Hamiltonian passes with shared partner loads and planner-chosen batch qubits, and
    first / last stages that read and write HBM directly next to ones that use the tile."""
    import oracle
    w = W.config(3, n=n, layers=layers)
    e_ref, g_ref = oracle.gradient_alg1(w.n, w.gates, w.theta, w.n_params, w.terms)
    with B.Circuit(w.n, w.gates, w.n_params, "c64", tile_qubits=13, specialize=2) as c:
        c.set_hamiltonian(w.terms)
        plan = c.plan()
        assert plan["tile_qubits"] == 13 and plan["specialized"] == 2
        e, g = c.energy_and_gradient(w.theta)
        assert_parity("c64", e, g, e_ref, g_ref, w.name)
        assert np.max(np.abs(c.get_state() - oracle.state(w.n, w.gates, w.theta))) <= 2e-5


@pytest.mark.gpu
def test_hamiltonian_plan_is_reproducible():
    """The Hamiltonian cover's randomised restarts use a fixed seed: two circuits planned
    from the same input get the same passes and bit-identical results."""
    w = W.config(3, n=20, layers=3)
    out = []
    for _ in range(2):
        with B.Circuit(w.n, w.gates, w.n_params, "c64", specialize=1) as c:
            c.set_hamiltonian(w.terms)
            out.append((c.plan()["hamiltonian_passes"],) + c.energy_and_gradient(w.theta))
    assert out[0][0] == out[1][0]
    assert out[0][1] == out[1][1] and np.array_equal(out[0][2], out[1][2])
