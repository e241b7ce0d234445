"""FP64 checkpoint norms and the invariants of the reverse sweep (Sec. 2.3: phi and lambda
are un-applied by the same unitaries, so <lambda_i|phi_{i+1}> = E and ||lambda_i|| stays
||H psi||), measured on the GPU by vqg_set_diagnostics / vqg_diagnostics at every forward
checkpoint and reverse restart, against the CPU oracle's E and ||H psi||^2."""
import numpy as np
import pytest

import oracle
from paper_2009_02823_gb300 import Circuit
from paper_2009_02823_gb300 import workloads as W
from tests.tolerances import TOL

pytestmark = pytest.mark.gpu


def _check(diag, e_ref, lam2_ref, dtype, n_ck_min):
    tol = TOL[dtype]
    assert diag["checkpoints"] >= n_ck_min
    assert abs(diag["energy"] - e_ref) <= tol * max(1.0, abs(e_ref))
    assert abs(diag["norm2_psi"] - 1.0) <= tol
    assert abs(diag["norm2_lambda"] - lam2_ref) <= tol * lam2_ref
    for d in diag["entries"]:
        assert d["stored"] == 1 and d["restarted"] == 1, d
        assert abs(d["norm2"] - 1.0) <= tol, d                            # ||psi_c|| = 1 (unitary sweep)
        assert abs(d["lam_phi_re"] - e_ref) <= tol * max(1.0, abs(e_ref)), d  # <lambda|phi> = E
        assert abs(d["lam_phi_im"]) <= tol * max(1.0, abs(e_ref)), d
        assert abs(d["norm2_lambda"] - lam2_ref) <= tol * lam2_ref, d      # ||lambda|| constant
        assert abs(d["norm2_unapplied"] - 1.0) <= tol, d
        assert d["drift2"] <= (1e-20 if dtype == "c128" else 1e-8), d    # what the restart replaces


def _reference(w):
    psi = oracle.state(w.n, w.gates, w.theta)
    lam = oracle.apply_hamiltonian(psi, w.terms)
    return float(np.real(np.vdot(psi, lam))), float(np.vdot(lam, lam).real)


@pytest.mark.parametrize("dtype,fusion,n,interval", [("c64", True, 12, 0), ("c128", True, 12, 40),
                                                     ("c64", False, 8, 16), ("c128", False, 8, 16)])
def test_invariants_small(dtype, fusion, n, interval):
    w = W.config(3, n=n, layers=6)
    e_ref, lam2_ref = _reference(w)
    with Circuit(w.n, w.gates, w.n_params, dtype, fusion=fusion, checkpoint_interval=interval) as c:
        c.set_hamiltonian(w.terms)
        e0, g0 = c.energy_and_gradient(w.theta)
        c.set_diagnostics(True)
        e1, g1 = c.energy_and_gradient(w.theta)
        diag = c.diagnostics()
        c.set_diagnostics(False)
        e2, g2 = c.energy_and_gradient(w.theta)
    assert e1 == e0 and np.array_equal(g1, g0)   # diagnostics change no result
    assert e2 == e0 and np.array_equal(g2, g0)
    _check(diag, e_ref, lam2_ref, dtype, 1)


def test_invariants_n24_bench_recipe():
    """The bench recipe (RY/RZ + CZ brickwork, 200 random Pauli strings) at n=24, complex64
    with the default checkpoints at every fused pass boundary."""
    w = W.config(3, n=24)
    e_ref, lam2_ref = _reference(w)
    with Circuit(w.n, w.gates, w.n_params, "c64") as c:
        c.set_hamiltonian(w.terms)
        c.set_diagnostics(True)
        c.energy_and_gradient(w.theta)
        diag = c.diagnostics()
        n_ck = c.plan()["checkpoints"]
    assert n_ck >= 3
    assert diag["checkpoints"] == n_ck
    _check(diag, e_ref, lam2_ref, "c64", n_ck)


def test_diagnostics_need_a_recorded_call():
    from paper_2009_02823_gb300 import binding as B
    w = W.config(1, n=6, layers=1)
    with Circuit(w.n, w.gates, w.n_params, "c64") as c:
        c.set_hamiltonian(w.terms)
        with pytest.raises(B.VqgError):
            c.diagnostics()
