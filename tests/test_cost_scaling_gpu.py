"""The paper's cost claim and a resource failure, on the GPU.

Sec. 2.3 / Fig. 2: the reverse-mode gradient (Algorithm 1) costs O(P) gate applications
while the faithful route (Algorithm 2, or parameter shift) costs O(P^2); the paper fits
straight lines to log runtime against log P.  Here both routes run on the GPU for the
RY/RZ + CZ brickwork at growing depth, and the fitted slopes must show the linear and the
quadratic growth (loose bounds: wall-clock timing).

A circuit whose state vectors do not fit the device is refused with VQG_ERR_OOM, and the
device stays usable."""
import time

import numpy as np
import pytest

from paper_2009_02823_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _slopes(n, layers):
    from paper_2009_02823_gb300 import Circuit
    P, t_adj, t_ps = [], [], []
    for L in layers:
        w = W.config(3, n=n, layers=L)
        with Circuit(w.n, w.gates, w.n_params, "c64") as c:
            # one diagonal term: the Hamiltonian pass (a cost independent of P) stays small
            c.set_hamiltonian([(1.0, ((0, "Z"), (n - 1, "Z")))])
            e0, g0 = c.energy_and_gradient(w.theta)
            reps = 10
            t0 = time.perf_counter()
            for _ in range(reps):
                c.energy_and_gradient(w.theta)
            t_adj.append((time.perf_counter() - t0) / reps)
            t0 = time.perf_counter()
            g_ps = c.gradient_parameter_shift(w.theta)
            t_ps.append(time.perf_counter() - t0)
            # both routes give the same gradient (complex64 bar)
            assert np.max(np.abs(g_ps - g0)) <= 1e-4 * max(np.max(np.abs(g0)), 1e-300)
        P.append(w.n_params)
    lp = np.log(P)
    return (float(np.polyfit(lp, np.log(t_adj), 1)[0]), float(np.polyfit(lp, np.log(t_ps), 1)[0]))


def test_adjoint_linear_parameter_shift_quadratic():
    # Costs independent of P (launch and host-sync latency, the Hamiltonian pass, the
    # reductions) flatten both curves at these small states, so the bounds sit below the
    # asymptotic slopes 1 and 2: the adjoint must not grow faster than linearly, the
    # parameter-shift gradient must grow clearly faster, by about one power of P.
    s_adj, s_ps = _slopes(20, (4, 8, 16, 32))
    print(f"log-log slopes in P: adjoint {s_adj:.3f}, parameter shift {s_ps:.3f}")
    assert s_adj <= 1.2, f"adjoint time grows faster than linearly in P (slope {s_adj:.2f})"
    assert 1.4 <= s_ps <= 2.3, f"parameter-shift slope {s_ps:.2f}"
    assert s_ps - s_adj >= 0.6, f"slopes {s_adj:.2f} / {s_ps:.2f}"


def test_out_of_memory_is_reported():
    from paper_2009_02823_gb300 import Circuit
    from paper_2009_02823_gb300.binding import VqgError
    n = 34  # complex128: 256 GiB per state, two states > the device's 280 GB
    gates = [("RY", q, -1, (q, -1, -1)) for q in range(n)]
    with pytest.raises(VqgError) as ei:
        Circuit(n, gates, n, "c128")
    assert ei.value.status == -2
    # the context is still usable
    w = W.config(3, n=12, layers=2)
    with Circuit(w.n, w.gates, w.n_params, "c64") as c:
        c.set_hamiltonian(w.terms)
        e, g = c.energy_and_gradient(w.theta)
        assert np.isfinite(e) and np.all(np.isfinite(g))
