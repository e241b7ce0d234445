"""Element-wise parity of the CUDA path (through the C ABI) with the CPU oracle on
seeded inputs: every gate kind at every qubit position (q = 0, 1, n-1 included),
repeated and multi-parameter gates, Pauli groups with Y factors, identity and
diagonal-only Hamiltonians, both precisions, the unfused and fused schedules, and
checkpointing."""
import numpy as np
import pytest

import oracle
from paper_2009_02823_gb300 import workloads as W
from tests.tolerances import TOL, assert_parity, energy_err, grad_err

pytestmark = pytest.mark.gpu

DTYPES = ["c128", "c64"]
MODES = [dict(fusion=False), dict(fusion=True)]


def _circ(w_n, gates, P, dtype, terms, **kw):
    from paper_2009_02823_gb300 import Circuit
    c = Circuit(w_n, gates, P, dtype, **kw)
    c.set_hamiltonian(terms)
    return c


def _oracle(n, gates, theta, P, terms):
    return oracle.gradient_alg1(n, gates, theta, P, terms)


@pytest.mark.parametrize("mode", MODES, ids=["per_gate", "fused"])
@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("seed", range(10))
def test_random_circuits(seed, dtype, mode):
    rng = np.random.default_rng(1000 + seed)
    n = [1, 2, 3, 4, 5, 7, 9, 11, 12, 13][seed]
    kinds = ("RX", "RY", "RZ", "U3") if n == 1 else ("RX", "RY", "RZ", "U3", "CNOT", "CZ")
    gates, P = W.random_circuit(rng, n, 40 + 4 * n, share_params=(seed % 3 == 0), kinds=kinds)
    theta = rng.uniform(0, 2 * np.pi, max(P, 1))[:P]
    terms = W.random_paulis(rng, n, 9, min(4, n))
    if seed == 4:
        terms.append((0.75, ()))  # identity term (x = z = 0)
    if seed == 5:
        terms = [(c, tuple((q, "Z") for q, _l in ops)) for c, ops in terms]  # diagonal only
    e_ref, g_ref = _oracle(n, gates, theta, P, terms)
    with _circ(n, gates, P, dtype, terms, **mode) as c:
        e, g = c.energy_and_gradient(theta)
        assert_parity(dtype, e, g, e_ref, g_ref, f"n={n}")
        assert energy_err(c.energy(theta), e_ref) <= TOL[dtype]
        psi = c.get_state()
        ref = oracle.state(n, gates, theta)
        assert np.max(np.abs(psi - ref)) <= (1e-12 if dtype == "c128" else 2e-5)


@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("kind", ["RX", "RY", "RZ", "U3", "CNOT", "CZ"])
def test_every_qubit_position(kind, dtype):
    """One gate kind on every qubit (and every ordered pair for entanglers), each with a
    preparing layer so no amplitude is trivially zero."""
    n = 6
    rng = np.random.default_rng(7)
    gates, P = [], 0
    for q in range(n):
        gates.append(("U3", q, -1, (P, P + 1, P + 2)))
        P += 3
    if kind in ("CNOT", "CZ"):
        for a in range(n):
            for b in range(n):
                if a != b:
                    gates.append((kind, a, b, (-1, -1, -1)))
                    gates.append(("RY", b, -1, (P, -1, -1)))
                    P += 1
    else:
        for q in range(n):
            k = 3 if kind == "U3" else 1
            gates.append((kind, q, -1, tuple(range(P, P + k)) + (-1,) * (3 - k)))
            P += k
            gates.append(("CNOT", q, (q + 1) % n, (-1, -1, -1)))
    theta = rng.uniform(0, 2 * np.pi, P)
    terms = W.random_paulis(rng, n, 12, 4)
    e_ref, g_ref = _oracle(n, gates, theta, P, terms)
    for mode in MODES:
        with _circ(n, gates, P, dtype, terms, **mode) as c:
            e, g = c.energy_and_gradient(theta)
            assert_parity(dtype, e, g, e_ref, g_ref, f"{kind} {mode}")


@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("mode", MODES, ids=["per_gate", "fused"])
def test_cfg1_vs_faithful_parameter_shift(dtype, mode):
    """n=10 hardware-efficient ansatz with TFIM: against the faithful O(P^2) oracle."""
    w = W.config(1)
    g_ref = oracle.gradient_parameter_shift(w.n, w.gates, w.theta, w.n_params, w.terms)
    e_ref = oracle.energy(w.n, w.gates, w.theta, w.terms)
    with _circ(w.n, w.gates, w.n_params, dtype, w.terms, **mode) as c:
        e, g = c.energy_and_gradient(w.theta)
        assert_parity(dtype, e, g, e_ref, g_ref, "cfg1")
        # repeated calls give bit-identical results (deterministic reductions)
        e2, g2 = c.energy_and_gradient(w.theta)
        assert e2 == e and np.array_equal(g2, g)


@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("cfg,n,layers", [(2, 12, 4), (3, 14, 3), (5, 10, 3), (1, 16, 2)])
def test_configs_reduced_size(cfg, n, layers, dtype):
    """Each workload recipe at a size the oracle finishes in seconds (several tiles and a
    ragged tail for the fused kernels)."""
    w = W.config(cfg, n=n, layers=layers)
    e_ref, g_ref = _oracle(w.n, w.gates, w.theta, w.n_params, w.terms)
    for mode in MODES:
        with _circ(w.n, w.gates, w.n_params, dtype, w.terms, **mode) as c:
            e, g = c.energy_and_gradient(w.theta)
            assert_parity(dtype, e, g, e_ref, g_ref, f"cfg{cfg} {mode}")


@pytest.mark.parametrize("dtype", DTYPES)
def test_gpu_parameter_shift_baseline(dtype):
    w = W.config(1, n=8, layers=2)
    g_ref = oracle.gradient_parameter_shift(w.n, w.gates, w.theta, w.n_params, w.terms)
    with _circ(w.n, w.gates, w.n_params, dtype, w.terms) as c:
        g = c.gradient_parameter_shift(w.theta)
        assert grad_err(g, g_ref) <= TOL[dtype]
        # a sub-range of occurrences
        g_part = c.gradient_parameter_shift(w.theta, 3, 9)
        ref_part = oracle.gradient_parameter_shift(w.n, w.gates, w.theta, w.n_params, w.terms, 3, 9)
        assert np.max(np.abs(g_part - ref_part)) <= TOL[dtype] * max(1.0, np.max(np.abs(ref_part)))


@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("interval", [1, 3, 7, 64])
def test_checkpoint_restarts(dtype, interval):
    """Forward-state checkpoints every `interval` gates (per-gate schedule) or at pass
    boundaries (fused schedule) restart phi in the reverse sweep; same gradient."""
    w = W.config(3, n=13, layers=4)
    e_ref, g_ref = _oracle(w.n, w.gates, w.theta, w.n_params, w.terms)
    for mode in MODES:
        with _circ(w.n, w.gates, w.n_params, dtype, w.terms, checkpoint_interval=interval,
                   tile_qubits=10, **mode) as c:
            info = c.plan()
            if mode["fusion"]:
                assert info["forward_passes"] > 1
                assert 1 <= info["checkpoints"] <= info["forward_passes"] - 1
            else:
                assert info["checkpoints"] == (w.n_gates - 1) // interval
            e, g = c.energy_and_gradient(w.theta)
            assert_parity(dtype, e, g, e_ref, g_ref, f"ckpt={interval} {mode}")


@pytest.mark.parametrize("dtype,K", [("c64", 10), ("c64", 11), ("c64", 12), ("c64", 13),
                                     ("c128", 10), ("c128", 11), ("c128", 12)])
@pytest.mark.parametrize("case", ["cfg2", "cfg3", "cfg5", "random"])
def test_fused_tile_sizes(case, dtype, K):
    """Every compiled tile size, with several tiles and several passes (n = 14)."""
    n = 14
    if case == "random":
        rng = np.random.default_rng(77 + K)
        gates, P = W.random_circuit(rng, n, 120, share_params=True)
        theta = rng.uniform(0, 2 * np.pi, P)
        terms = W.random_paulis(rng, n, 25, 4)
    else:
        w = W.config(int(case[3]), n=n, layers=3)
        gates, P, theta, terms = w.gates, w.n_params, w.theta, w.terms
    e_ref, g_ref = _oracle(n, gates, theta, P, terms)
    with _circ(n, gates, P, dtype, terms, tile_qubits=K) as c:
        info = c.plan()
        assert info["tile_qubits"] == K and info["forward_passes"] >= 1
        e, g = c.energy_and_gradient(theta)
        assert_parity(dtype, e, g, e_ref, g_ref, f"{case} K={K}")
        assert energy_err(c.energy(theta), e_ref) <= TOL[dtype]
        psi = c.get_state()
        assert np.max(np.abs(psi - oracle.state(n, gates, theta))) <= (1e-12 if dtype == "c128" else 2e-5)


def test_hamiltonian_can_change_between_calls():
    w = W.config(1, n=9, layers=2)
    rng = np.random.default_rng(3)
    with _circ(w.n, w.gates, w.n_params, "c128", w.terms) as c:
        for _ in range(3):
            terms = W.random_paulis(rng, w.n, 7, 3)
            c.set_hamiltonian(terms)
            e_ref, g_ref = _oracle(w.n, w.gates, w.theta, w.n_params, terms)
            e, g = c.energy_and_gradient(w.theta)
            assert_parity("c128", e, g, e_ref, g_ref, "H swap")


def test_empty_and_degenerate():
    """No gates; no parameters; empty Hamiltonian; one qubit."""
    from paper_2009_02823_gb300 import Circuit
    with Circuit(3, [], 0, "c128") as c:
        c.set_hamiltonian([(1.0, ((0, "Z"),)), (0.5, ((1, "X"),))])
        e, g = c.energy_and_gradient(np.zeros(0))
        assert e == pytest.approx(1.0, abs=1e-15) and g.size == 0
    with Circuit(2, [("CNOT", 0, 1, (-1, -1, -1))], 0, "c64") as c:
        c.set_hamiltonian([])
        e, g = c.energy_and_gradient(np.zeros(0))
        assert e == 0.0
    with Circuit(1, [("RX", 0, -1, (0, -1, -1))], 1, "c128") as c:
        c.set_hamiltonian([(1.0, ((0, "Z"),))])
        for t in (0.0, 0.4, np.pi, 5.0):
            e, g = c.energy_and_gradient(np.array([t]))
            assert e == pytest.approx(np.cos(t), abs=1e-14)
            assert g[0] == pytest.approx(-np.sin(t), abs=1e-14)


def test_unused_parameter_has_zero_gradient():
    from paper_2009_02823_gb300 import Circuit
    gates = [("RY", 0, -1, (2, -1, -1)), ("CNOT", 0, 1, (-1, -1, -1)), ("RX", 1, -1, (0, -1, -1))]
    th = np.array([0.3, 1.7, 0.9])
    terms = [(1.0, ((0, "Z"), (1, "Z"))), (0.3, ((1, "X"),))]
    e_ref, g_ref = _oracle(2, gates, th, 3, terms)
    with Circuit(2, gates, 3, "c128") as c:
        c.set_hamiltonian(terms)
        e, g = c.energy_and_gradient(th)
        assert g[1] == 0.0
        assert_parity("c128", e, g, e_ref, g_ref)


@pytest.mark.parametrize("dtype,K,Rf,Rr", [("c64", 12, 4, 3), ("c64", 13, 4, 4), ("c64", 10, 5, 3),
                                           ("c128", 11, 3, 2), ("c128", 12, 3, 3), ("c128", 10, 4, 2)])
@pytest.mark.parametrize("case", ["cfg3", "cfg5", "random"])
def test_fused_register_variants(case, dtype, K, Rf, Rr):
    """Every compiled register-qubit variant of the fused passes against the oracle."""
    n = 14
    if case == "random":
        rng = np.random.default_rng(99 + K + Rf)
        gates, P = W.random_circuit(rng, n, 120, share_params=True)
        theta = rng.uniform(0, 2 * np.pi, P)
        terms = W.random_paulis(rng, n, 25, 4)
    else:
        w = W.config(int(case[3]), n=n, layers=3)
        gates, P, theta, terms = w.gates, w.n_params, w.theta, w.terms
    e_ref, g_ref = _oracle(n, gates, theta, P, terms)
    with _circ(n, gates, P, dtype, terms, tile_qubits=K, fwd_reg_qubits=Rf, rev_reg_qubits=Rr) as c:
        e, g = c.energy_and_gradient(theta)
        assert_parity(dtype, e, g, e_ref, g_ref, f"{case} K={K} R=({Rf},{Rr})")


@pytest.mark.parametrize("dtype", DTYPES)
def test_cuda_graph_replay(dtype):
    """use_graph: the captured launch sequence replays with new theta values."""
    import torch
    w = W.config(3, n=13, layers=3)
    s = torch.cuda.Stream()
    with _circ(w.n, w.gates, w.n_params, dtype, w.terms, use_graph=True, stream=s) as c:
        rng = np.random.default_rng(8)
        for k in range(4):
            th = w.theta if k == 0 else rng.uniform(0, 2 * np.pi, w.n_params)
            e_ref, g_ref = _oracle(w.n, w.gates, th, w.n_params, w.terms)
            e, g = c.energy_and_gradient(th)
            assert_parity(dtype, e, g, e_ref, g_ref, f"graph call {k}")


@pytest.mark.parametrize("dtype", DTYPES)
def test_autotune_choice_and_parity(dtype):
    """The autotuner times candidate schedules, keeps a compiled one, stores it in the
    process-wide table (a second circuit of the same structure reuses it untimed), and
    the tuned circuit still matches the oracle.  options.autotune runs it on the first
    evaluation."""
    from paper_2009_02823_gb300 import binding as B
    B.lib().vqg_tune_table_clear()
    w = W.config(2, n=16, layers=3)
    e_ref, g_ref = _oracle(w.n, w.gates, w.theta, w.n_params, w.terms)
    kmax = 13 if dtype == "c64" else 12
    with _circ(w.n, w.gates, w.n_params, dtype, w.terms) as c:
        r = c.autotune(w.theta)
        assert r["candidates"] >= 3 and kmax - 2 <= r["tile_qubits"] <= kmax
        assert 0 < r["best_ms"] and r["default_ms"] > 0
        info = c.plan()
        assert (info["tile_qubits"], info["fwd_reg_qubits"], info["rev_reg_qubits"]) == \
            (r["tile_qubits"], r["fwd_reg_qubits"], r["rev_reg_qubits"])
        e, g = c.energy_and_gradient(w.theta)
        assert_parity(dtype, e, g, e_ref, g_ref, "tuned")
    with _circ(w.n, w.gates, w.n_params, dtype, w.terms, autotune=True) as c:
        e, g = c.energy_and_gradient(w.theta)  # tunes first (from the table)
        assert_parity(dtype, e, g, e_ref, g_ref, "autotune option")
        r2 = c.autotune(w.theta)
        assert r2["candidates"] == 0 and r2["tile_qubits"] == r["tile_qubits"]
        assert c.plan()["tile_qubits"] == r["tile_qubits"]
    with _circ(w.n, w.gates, w.n_params, dtype, w.terms, tile_qubits=11) as c:
        r3 = c.autotune(w.theta)  # explicit tile: nothing to tune
        assert r3["candidates"] == 0 and c.plan()["tile_qubits"] == 11


# ---------------------------------------------------------------- controlled rotations and phase gates (App. A)
ALL_KINDS = ("RX", "RY", "RZ", "U3", "CNOT", "CZ", "CRX", "CRY", "CRZ", "PHASE", "CPHASE")


@pytest.mark.parametrize("mode", MODES, ids=["per_gate", "fused"])
@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("seed", range(8))
def test_controlled_random_circuits(seed, dtype, mode):
    rng = np.random.default_rng(2000 + seed)
    n = [2, 3, 5, 7, 10, 11, 12, 13][seed]
    gates, P = W.random_circuit(rng, n, 50 + 5 * n, share_params=(seed % 3 == 0), kinds=ALL_KINDS)
    theta = rng.uniform(0, 2 * np.pi, max(P, 1))[:P]
    terms = W.random_paulis(rng, n, 9, min(4, n))
    e_ref, g_ref = _oracle(n, gates, theta, P, terms)
    with _circ(n, gates, P, dtype, terms, **mode) as c:
        e, g = c.energy_and_gradient(theta)
        assert_parity(dtype, e, g, e_ref, g_ref, f"n={n}")
        assert energy_err(c.energy(theta), e_ref) <= TOL[dtype]  # forward sweep only: psi = U|0>
        psi = c.get_state()
        assert np.max(np.abs(psi - oracle.state(n, gates, theta))) <= (1e-12 if dtype == "c128" else 2e-5)


@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("kind", ["CRX", "CRY", "CRZ", "PHASE", "CPHASE"])
@pytest.mark.parametrize("n", [6, 11])
def test_controlled_every_position(kind, dtype, n):
    """Each new kind on every (control, target) pair (every qubit for PHASE) after a
    U3 layer, fused (n = 11) and per gate (n = 6): controls on register, thread-level
    and tile-external bits all occur in the fused case."""
    rng = np.random.default_rng(17)
    gates, P = [], 0
    for q in range(n):
        gates.append(("U3", q, -1, (P, P + 1, P + 2)))
        P += 3
    pairs = [(q, -1) for q in range(n)] if kind == "PHASE" else \
        [(a, b) for a in range(n) for b in range(n) if a != b]
    for a, b in pairs:
        gates.append((kind, a, b, (P, -1, -1)))
        P += 1
        if len(gates) % 7 == 0:
            gates.append(("RY", int(rng.integers(0, n)), -1, (P, -1, -1)))
            P += 1
    theta = rng.uniform(0, 2 * np.pi, P)
    terms = W.random_paulis(rng, n, 12, 4)
    e_ref, g_ref = _oracle(n, gates, theta, P, terms)
    with _circ(n, gates, P, dtype, terms) as c:
        e, g = c.energy_and_gradient(theta)
        assert_parity(dtype, e, g, e_ref, g_ref, f"{kind} n={n}")


@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("K", [10, 11, 12])
def test_controlled_fused_tile_sizes(dtype, K):
    """The controlled-rotation ansatz (Circuit D-like ring) at n = 14 under several tile
    sizes and both register widths, against the oracle."""
    n = 14
    gates, P = W.crx_ring(n, 4)
    rng = np.random.default_rng(5)
    theta = rng.uniform(0, 2 * np.pi, P)
    terms = W.random_paulis(rng, n, 20, 4)
    e_ref, g_ref = _oracle(n, gates, theta, P, terms)
    regs = ((5, 4), (4, 3)) if dtype == "c64" else ((4, 3), (3, 2))
    for Rf, Rr in regs:
        if Rr == 2 and K > 11:
            continue
        with _circ(n, gates, P, dtype, terms, tile_qubits=K, fwd_reg_qubits=Rf, rev_reg_qubits=Rr) as c:
            e, g = c.energy_and_gradient(theta)
            assert_parity(dtype, e, g, e_ref, g_ref, f"K={K} R={Rf}/{Rr}")


@pytest.mark.parametrize("dtype", DTYPES)
def test_gpu_parameter_shift_controlled(dtype):
    """The GPU parameter-shift baseline with the four-term rule of controlled rotations
    agrees with the oracle's Algorithm-1 gradient (an independent route)."""
    n = 6
    gates, P = W.crx_ring(n, 2)
    gates = gates + [("PHASE", 2, -1, (P, -1, -1)), ("CPHASE", 0, 4, (P + 1, -1, -1)),
                     ("CRY", 3, 1, (P + 2, -1, -1)), ("CRZ", 5, 0, (P + 3, -1, -1))]
    P += 4
    rng = np.random.default_rng(8)
    theta = rng.uniform(0, 2 * np.pi, P)
    terms = W.random_paulis(rng, n, 10, 3)
    _e, g_ref = _oracle(n, gates, theta, P, terms)
    with _circ(n, gates, P, dtype, terms) as c:
        assert grad_err(c.gradient_parameter_shift(theta), g_ref) <= TOL[dtype]


# ---------------------------------------------------------------- non-Hermitian operators (App. B.4)
def _assert_complex_parity(dtype, e, g, e_ref, g_ref, what):
    scale = max(float(np.max(np.abs(g_ref))) if len(g_ref) else 0.0, 1e-300)
    assert abs(e - e_ref) <= TOL[dtype] * max(1.0, abs(e_ref)), (what, e, e_ref)
    if len(g_ref):
        assert float(np.max(np.abs(g - g_ref))) / scale <= TOL[dtype], (what, float(np.max(np.abs(g - g_ref))))


def _complex_terms(rng, n, count):
    return [(complex(c, float(rng.normal())), ops) for c, ops in W.random_paulis(rng, n, count, min(4, n))]


@pytest.mark.parametrize("mode", MODES, ids=["per_gate", "fused"])
@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("seed", range(6))
def test_non_hermitian_random(seed, dtype, mode):
    rng = np.random.default_rng(3000 + seed)
    n = [2, 4, 7, 10, 12, 13][seed]
    gates, P = W.random_circuit(rng, n, 40 + 4 * n, share_params=(seed % 2 == 0), kinds=ALL_KINDS)
    theta = rng.uniform(0, 2 * np.pi, max(P, 1))[:P]
    terms = _complex_terms(rng, n, 10)
    if seed == 3:
        terms = [(1j * abs(c), ops) for c, ops in terms]  # purely anti-Hermitian
    e_ref, g_ref = oracle.gradient_alg1_operator(n, gates, theta, P, terms)
    from paper_2009_02823_gb300 import Circuit
    with Circuit(n, gates, P, dtype, **mode) as c:
        c.set_operator(terms)
        for _ in range(2):  # repeated calls reuse both parts' plans
            e, g = c.expectation_and_gradient(theta)
            _assert_complex_parity(dtype, e, g, e_ref, g_ref, f"n={n}")


def test_non_hermitian_modes_and_errors():
    """A Hermitian operator through set_operator (imaginary parts 0), the refusal of the
    real entry points while the operator is not Hermitian, set_hamiltonian restoring
    Hermitian mode, the device entry point, and an empty Hamiltonian (gradient 0)."""
    from paper_2009_02823_gb300 import Circuit
    from paper_2009_02823_gb300.binding import VqgError
    import torch
    rng = np.random.default_rng(31)
    w = W.config(1, n=11, layers=2)
    with Circuit(w.n, w.gates, w.n_params, "c128") as c:
        c.set_operator(w.terms)
        e, g = c.expectation_and_gradient(w.theta)
        e_ref, g_ref = oracle.gradient_alg1(w.n, w.gates, w.theta, w.n_params, w.terms)
        _assert_complex_parity("c128", e, g, complex(e_ref), g_ref.astype(complex), "hermitian via set_operator")
        terms = _complex_terms(rng, w.n, 8)
        c.set_operator(terms)
        with pytest.raises(VqgError) as ei:
            c.energy_and_gradient(w.theta)
        assert ei.value.status == -6
        e_ref, g_ref = oracle.gradient_alg1_operator(w.n, w.gates, w.theta, w.n_params, terms)
        th = torch.tensor(w.theta, dtype=torch.float64, device="cuda")
        ed = torch.zeros(2, dtype=torch.float64, device="cuda")
        gd = torch.zeros(2 * w.n_params, dtype=torch.float64, device="cuda")
        c.expectation_and_gradient_device(th.data_ptr(), ed.data_ptr(), gd.data_ptr())
        torch.cuda.synchronize()
        e = complex(float(ed[0]), float(ed[1]))
        g = gd.cpu().numpy()
        _assert_complex_parity("c128", e, g[0::2] + 1j * g[1::2], e_ref, g_ref, "device entry point")
        c.set_hamiltonian(w.terms)
        e, g = c.energy_and_gradient(w.theta)
        e_ref, g_ref = oracle.gradient_alg1(w.n, w.gates, w.theta, w.n_params, w.terms)
        assert_parity("c128", e, g, e_ref, g_ref, "set_hamiltonian after set_operator")
        c.set_hamiltonian([])
        e, g = c.energy_and_gradient(w.theta)
        assert e == 0.0 and np.all(g == 0.0)


@pytest.mark.parametrize("dtype", DTYPES)
def test_non_hermitian_after_autotune(dtype):
    """The autotuner re-plans both operator parts."""
    from paper_2009_02823_gb300 import Circuit
    rng = np.random.default_rng(41)
    w = W.config(2, n=15, layers=2)
    terms = _complex_terms(rng, w.n, 12)
    e_ref, g_ref = oracle.gradient_alg1_operator(w.n, w.gates, w.theta, w.n_params, terms)
    with Circuit(w.n, w.gates, w.n_params, dtype) as c:
        c.set_operator(terms)
        c.autotune(w.theta)
        e, g = c.expectation_and_gradient(w.theta)
        _assert_complex_parity(dtype, e, g, e_ref, g_ref, "tuned")


# ---------------------------------------------------------------- tensor-product operators and input states
HAD = np.array([[1, 1], [1, -1]], dtype=complex) / np.sqrt(2)


def _rand_herm(rng):
    a = rng.normal(size=(2, 2)) + 1j * rng.normal(size=(2, 2))
    return (a + a.conj().T) / 2


@pytest.mark.parametrize("mode", MODES, ids=["per_gate", "fused"])
@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("seed", range(6))
def test_products_and_input_state(seed, dtype, mode):
    """Sums of tensor products (Hadamard^N and random Hermitian factors), with and
    without a random input state, against the oracle's general Algorithm-1 route."""
    from paper_2009_02823_gb300 import Circuit
    rng = np.random.default_rng(4000 + seed)
    n = [3, 6, 10, 11, 12, 13][seed]
    gates, P = W.random_circuit(rng, n, 30 + 3 * n, share_params=(seed % 2 == 1), kinds=ALL_KINDS)
    theta = rng.uniform(0, 2 * np.pi, max(P, 1))[:P]
    products = [(1.0, [HAD] * n)] + [(float(rng.normal()), [_rand_herm(rng) for _ in range(n)])
                                     for _ in range(seed % 3)]
    psi0 = None
    if seed % 2 == 0:
        psi0 = rng.normal(size=1 << n) + 1j * rng.normal(size=1 << n)
        psi0 /= np.linalg.norm(psi0)
    e_ref, g_ref = oracle.gradient_general("alg1", n, gates, theta, P, products=products, in_state=psi0)
    with Circuit(n, gates, P, dtype, **mode) as c:
        c.set_product_operator(products)
        if psi0 is not None:
            c.set_input_state(psi0)
        for _ in range(2):
            e, g = c.energy_and_gradient(theta)
            assert_parity(dtype, e, g, e_ref, g_ref, f"n={n} products={len(products)}")
        assert energy_err(c.energy(theta), e_ref) <= TOL[dtype]
        if psi0 is not None:  # back to |0...0>
            c.set_input_state(None)
            e_ref0, g_ref0 = oracle.gradient_general("alg1", n, gates, theta, P, products=products)
            e, g = c.energy_and_gradient(theta)
            assert_parity(dtype, e, g, e_ref0, g_ref0, "input cleared")
        c.set_hamiltonian(W.random_paulis(rng, n, 5, min(4, n)))  # Pauli Hamiltonian again
        c.energy_and_gradient(theta)


def test_product_operator_rejects_non_hermitian():
    from paper_2009_02823_gb300 import Circuit
    from paper_2009_02823_gb300.binding import VqgError
    gates, P = W.hea_ry_rz(4, 1)
    with Circuit(4, gates, P, "c64") as c:
        with pytest.raises(VqgError) as ei:
            c.set_product_operator([(1.0, [np.array([[0, 1], [0, 0]])] * 4)])
        assert ei.value.status == -5


@pytest.mark.parametrize("dtype", DTYPES)
def test_hadamard_product_full_size_closed_form(dtype):
    """Hadamard^{(x)30} on an RY layer over 30 qubits (8 / 16 GiB states): E and every
    gradient entry against the closed form prod_q f(t_q), f = (sin t + cos t)/sqrt2."""
    from paper_2009_02823_gb300 import Circuit
    n = 30
    rng = np.random.default_rng(30)
    t = np.pi / 4 + 0.2 * rng.normal(size=n)
    gates = [("RY", q, -1, (q, -1, -1)) for q in range(n)]
    f = (np.sin(t) + np.cos(t)) / np.sqrt(2)
    df = (np.cos(t) - np.sin(t)) / np.sqrt(2)
    e_ref = float(np.prod(f))
    g_ref = np.array([df[q] * np.prod(np.delete(f, q)) for q in range(n)])
    with Circuit(n, gates, n, dtype) as c:
        c.set_product_operator([(1.0, [HAD] * n)])
        e, g = c.energy_and_gradient(t)
        assert_parity(dtype, e, g, e_ref, g_ref, "H^30")


@pytest.mark.parametrize("theta0", [np.pi / 2, np.pi / 2 + 1e-6, 3 * np.pi / 2, np.pi / 2 - 3e-7])
def test_long_scaled_ry_stages(theta0):
    """complex64 RY ops run in a scaled form whose dropped factors |k| >= 2^-1/2 multiply up
    over a register stage; theta = pi/2 (+-) makes every |k| = 2^-1/2, the largest total
    scale.  Long runs of RY on the low qubits (register qubits of the tile passes) with a
    CZ ladder between runs, against the oracle at the complex64 bar."""
    n = 12
    rng = np.random.default_rng(31)
    gates, P = [], 0
    for q in range(n):  # a random preparing layer, so that no gradient entry vanishes by symmetry
        gates.append(("RX", q, -1, (P, -1, -1)))
        gates.append(("RZ", q, -1, (P + 1, -1, -1)))
        P += 2
    n_prep = P
    for rep in range(12):
        for q in range(6):
            gates.append(("RY", q, -1, (P, -1, -1)))
            P += 1
        if rep % 3 == 2:
            for q in range(0, n - 1, 2):
                gates.append(("CZ", q, q + 1, (-1, -1, -1)))
    theta = np.full(P, theta0) + rng.uniform(-1e-7, 1e-7, P) * (theta0 != np.pi / 2)
    theta[:n_prep] = rng.uniform(0, 2 * np.pi, n_prep)
    terms = W.random_paulis(rng, n, 12, 4)
    e_ref, g_ref = _oracle(n, gates, theta, P, terms)
    with _circ(n, gates, P, "c64", terms) as c:
        assert c.plan()["tile_qubits"] > 0
        e, g = c.energy_and_gradient(theta)
        assert_parity("c64", e, g, e_ref, g_ref, f"theta0={theta0}")


@pytest.mark.parametrize("K", [10, 12])
def test_hamiltonian_without_diagonal_terms(K):
    """Every term flips a qubit, so the diagonal (x = 0) group exists but holds no term;
    one group mixes a real-weight and an imaginary-weight term (X3 and Y3).  K = n puts
    the whole state in one tile."""
    n = 12
    rng = np.random.default_rng(5)
    gates, P = W.random_circuit(rng, n, 60, share_params=False)
    theta = rng.uniform(0, 2 * np.pi, P)
    terms = [(c, ops) for c, ops in W.random_paulis(rng, n, 14, 4) if any(l in "XY" for _q, l in ops)]
    terms += [(-0.23, ((3, "X"),)), (1.31, ((3, "Y"),)), (0.7, ((1, "X"), (5, "Z"))), (0.4, ((1, "Y"), (5, "Y")))]
    e_ref, g_ref = _oracle(n, gates, theta, P, terms)
    for dtype in DTYPES:
        with _circ(n, gates, P, dtype, terms, tile_qubits=K) as c:
            e, g = c.energy_and_gradient(theta)
            assert_parity(dtype, e, g, e_ref, g_ref, f"K={K}")
            assert energy_err(c.energy(theta), e_ref) <= TOL[dtype]
