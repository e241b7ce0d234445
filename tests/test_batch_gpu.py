"""The batched persistent launch: parity with the oracle on a small batch of uneven
circuits, agreement with single-circuit evaluations on the full 512-circuit recipe,
graph replay with new parameters, and the bounded-wait error path."""
import numpy as np
import pytest

import oracle
from paper_2009_02823_gb300 import workloads as W
from tests.tolerances import TOL, assert_parity, grad_err

pytestmark = pytest.mark.gpu


def _small_batch():
    ws = W.batched(count=6, nmin=12, nmax=14, dmin=2, dmax=4, seed_cfg=41)
    rng = np.random.default_rng(12)
    gates, P = W.random_circuit(rng, 13, 60, share_params=True)
    ws.append(W.Workload("random13", 13, gates, P, rng.uniform(0, 2 * np.pi, P), W.random_paulis(rng, 13, 20, 4)))
    w5 = W.config(5, n=12, layers=2)
    ws.append(w5)
    return ws


def test_small_batch_vs_oracle():
    from paper_2009_02823_gb300.batch import Batch
    ws = _small_batch()
    with Batch(ws) as b:
        for call in range(3):  # eager, captured, replayed
            thetas = [w.theta + 0.1 * call for w in ws]
            e, g = b.energy_and_gradient(thetas)
            for k, w in enumerate(ws):
                e_ref, g_ref = oracle.gradient_alg1(w.n, w.gates, thetas[k], w.n_params, w.terms)
                assert_parity("c64", e[k], g[k], e_ref, g_ref, f"batch circuit {k} call {call}")


def test_batch_autotune_then_parity():
    """The geometry autotuner times both compiled tile geometries, keeps one, and the
    batch still matches the oracle afterwards (eager, captured and replayed calls)."""
    from paper_2009_02823_gb300.batch import Batch
    ws = _small_batch()
    with Batch(ws) as b:
        b.energy_and_gradient([w.theta for w in ws])  # built and run before tuning
        r = b.autotune([w.theta for w in ws])
        assert r["candidates"] == 2 and (r["tile_qubits"], r["fwd_reg_qubits"]) in ((12, 4), (11, 3))
        assert r["best_ms"] > 0 and r["default_ms"] >= r["best_ms"]
        for call in range(3):
            thetas = [w.theta - 0.05 * call for w in ws]
            e, g = b.energy_and_gradient(thetas)
            for k, w in enumerate(ws):
                e_ref, g_ref = oracle.gradient_alg1(w.n, w.gates, thetas[k], w.n_params, w.terms)
                assert_parity("c64", e[k], g[k], e_ref, g_ref, f"tuned batch circuit {k} call {call}")


def test_batch_both_geometries_match_oracle():
    """Both compiled tile geometries give oracle results, whatever the tuner picks."""
    from paper_2009_02823_gb300 import binding as B
    from paper_2009_02823_gb300.batch import Batch
    ws = _small_batch()[:4]
    with Batch(ws) as b:
        for K in (11, 12):
            b.set_tile_qubits(K)
            e, g = b.energy_and_gradient([w.theta for w in ws])
            for k, w in enumerate(ws):
                e_ref, g_ref = oracle.gradient_alg1(w.n, w.gates, w.theta, w.n_params, w.terms)
                assert_parity("c64", e[k], g[k], e_ref, g_ref, f"tile qubits {K} circuit {k}")
        with pytest.raises(B.VqgError):
            b.set_tile_qubits(13)


def test_wait_timeout_is_reported_and_recoverable():
    from paper_2009_02823_gb300.batch import Batch
    from paper_2009_02823_gb300.binding import VqgError
    ws = _small_batch()[:3]
    with Batch(ws) as b:
        b.set_wait_limit(20000, stall_circuit=1)  # circuit 1's later phases never become ready
        with pytest.raises(VqgError) as ei:
            b.energy_and_gradient([w.theta for w in ws])
        assert ei.value.status == -4
        b.set_wait_limit(1 << 26, stall_circuit=-1)
        e, g = b.energy_and_gradient([w.theta for w in ws])
        for k, w in enumerate(ws):
            e_ref, g_ref = oracle.gradient_alg1(w.n, w.gates, w.theta, w.n_params, w.terms)
            assert_parity("c64", e[k], g[k], e_ref, g_ref, f"after timeout, circuit {k}")


def test_full_recipe_512_circuits():
    """512 circuits, n in 12..20, 4..16 layers: sampled circuits agree with the
    single-circuit complex64 path and the smallest ones with the oracle."""
    from paper_2009_02823_gb300 import Circuit
    from paper_2009_02823_gb300.batch import Batch
    ws = W.batched()
    with Batch(ws) as b:
        info = b.info()
        assert info["total_params"] == sum(w.n_params for w in ws)
        e, g = b.energy_and_gradient([w.theta for w in ws])
        e2, g2 = b.energy_and_gradient([w.theta for w in ws])
    assert np.array_equal(e, e2)  # deterministic
    rng = np.random.default_rng(4)
    for k in rng.choice(len(ws), 12, replace=False):
        w = ws[k]
        with Circuit(w.n, w.gates, w.n_params, "c64") as c:
            c.set_hamiltonian(w.terms)
            es, gs = c.energy_and_gradient(w.theta)
        assert abs(e[k] - es) <= TOL["c64"] * max(1.0, abs(es))
        assert grad_err(g[k], gs) <= TOL["c64"]
    small = [k for k, w in enumerate(ws) if w.n == 12][:3]
    for k in small:
        w = ws[k]
        e_ref, g_ref = oracle.gradient_alg1(w.n, w.gates, w.theta, w.n_params, w.terms)
        assert_parity("c64", e[k], g[k], e_ref, g_ref, f"recipe circuit {k}")


def test_batch_with_controlled_gates():
    """Circuits with controlled rotations and phase gates run through the batched launch
    (both tile geometries) and match the oracle."""
    from paper_2009_02823_gb300.batch import Batch
    rng = np.random.default_rng(77)
    ws = []
    for k in range(4):
        n = 12 + k % 2
        kinds = ("RX", "RY", "RZ", "CNOT", "CZ", "CRX", "CRY", "CRZ", "PHASE", "CPHASE")
        gates, P = W.random_circuit(rng, n, 80, share_params=(k == 1), kinds=kinds)
        ws.append(W.Workload(f"ctl{k}", n, gates, P, rng.uniform(0, 2 * np.pi, P), W.random_paulis(rng, n, 10, 4)))
    gates, P = W.crx_ring(12, 3)
    ws.append(W.Workload("ring12", 12, gates, P, rng.uniform(0, 2 * np.pi, P), W.tfim(12, 0.8)))
    with Batch(ws) as b:
        for K in (12, 11):
            b.set_tile_qubits(K)
            e, g = b.energy_and_gradient([w.theta for w in ws])
            for k, w in enumerate(ws):
                e_ref, g_ref = oracle.gradient_alg1(w.n, w.gates, w.theta, w.n_params, w.terms)
                assert_parity("c64", e[k], g[k], e_ref, g_ref, f"K={K} circuit {k}")
