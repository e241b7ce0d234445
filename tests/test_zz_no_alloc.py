"""vqg_reverse_noalloc, the entry point that allocates nothing, checked against the
regular vqg_energy_and_gradient on the same circuit and against the CPU oracle's
Algorithm 1 gradient.

Callers that may not allocate device memory while they run (a framework's caching
pool owns the GPU, the footprint is fixed at start-up, or a latency-critical thread
must not enter cudaMalloc/cudaFree) hand the library their own state vectors; the
reduction scratch lives in static device arrays.  This file is collected last so that
a failure here leaves every other test already run.
"""
import numpy as np
import pytest

import oracle
from paper_2009_02823_gb300 import binding as B
from paper_2009_02823_gb300 import workloads as W
from tests.tolerances import TOL, grad_err


def _case():
    rng = np.random.default_rng(4242)
    n = 11
    gates, P = W.random_circuit(rng, n, 70, share_params=True)
    theta = rng.uniform(0, 2 * np.pi, P)
    terms = W.random_paulis(rng, n, 10, 4)
    return n, gates, P, theta, terms


@pytest.mark.parametrize("kind", ["CRX", "CRY", "CRZ", "PHASE", "CPHASE"])
def test_rejects_controlled_and_phase_gates(kind):
    gate = (kind, 0, 1, (0, -1, -1)) if kind != "PHASE" else (kind, 0, -1, (0, -1, -1))
    with pytest.raises(B.VqgError) as ei:
        B.reverse_noalloc(3, "c64", [gate], np.zeros(1), 1, 1, 1, 1)
    assert ei.value.status == -1 and "RX, RY, RZ, U3, CNOT and CZ" in str(ei.value)


def test_rejects_too_many_gates():
    n, gates, P, theta, _terms = _case()
    big = gates[: B.NOALLOC_MAX_GATES + 1]
    assert len(big) == B.NOALLOC_MAX_GATES + 1
    with pytest.raises(B.VqgError) as ei:
        B.reverse_noalloc(n, "c64", big, theta, P, 1, 1, 1)
    assert ei.value.status == -1 and "at most" in str(ei.value)


@pytest.mark.gpu
@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_noalloc_matches_energy_and_gradient(dtype):
    import torch

    n, gates, P, theta, terms = _case()
    with B.Circuit(n, gates, P, dtype) as c:
        c.set_hamiltonian(terms)
        e_ref, g_ref = c.energy_and_gradient(theta)
    # psi and lambda = H psi as the reverse sweep starts (Algorithm 1, before the reverse loop)
    psi = oracle.state(n, gates, theta)
    lam = oracle.apply_hamiltonian(psi, terms)
    e_or, g_or = oracle.gradient_alg1(n, gates, theta, P, terms)
    cdt = torch.complex64 if dtype == "c64" else torch.complex128
    stream = torch.cuda.current_stream()
    segments = [gates[i:i + B.NOALLOC_MAX_GATES] for i in range(0, len(gates), B.NOALLOC_MAX_GATES)]
    assert len(segments) >= 2
    results = []
    for _repeat in range(2):  # two full sweeps in a row share the static scratch
        phi_d = torch.tensor(psi, dtype=cdt, device="cuda")
        lam_d = torch.tensor(lam, dtype=cdt, device="cuda")
        grad_d = torch.zeros(P, dtype=torch.float64, device="cuda")
        tol = 1e-12 if dtype == "c128" else 2e-5
        nl = float(np.linalg.norm(lam))
        for seg in reversed(segments):  # last segment first, one call per segment
            B.reverse_noalloc(n, dtype, seg, theta, P, phi_d.data_ptr(), lam_d.data_ptr(),
                              grad_d.data_ptr(), stream)
            torch.cuda.synchronize()
            # invariants of the recurrence (Sec. 2.2): both vectors are un-applied by the same
            # unitaries, so <lambda_i|phi_{i+1}> stays E and the norms stay put
            f, l_ = phi_d.cpu().numpy(), lam_d.cpu().numpy()
            assert abs(np.vdot(l_, f) - e_ref) <= tol * max(1.0, abs(e_ref))
            assert abs(np.linalg.norm(f) - 1.0) <= tol
            assert abs(np.linalg.norm(l_) - nl) <= tol * max(1.0, nl)
        g = grad_d.cpu().numpy()
        assert grad_err(g, g_ref) <= TOL[dtype], grad_err(g, g_ref)
        assert grad_err(g, g_or) <= TOL[dtype], grad_err(g, g_or)
        # phi has been swept back to the input state |0...0>
        phi_end = phi_d.cpu().numpy()
        assert abs(phi_end[0]) == pytest.approx(1.0, abs=1e-10 if dtype == "c128" else 1e-5)
        results.append(g)
    assert np.array_equal(results[0], results[1])
