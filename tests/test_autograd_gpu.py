"""The torch.autograd wrapper: gradients from backward() equal the library's
reverse-mode gradient, the oracle, and central finite differences (Eq. 2, symmetric
form, delta = 1e-4 in FP64); host and device theta; an Adam loop on the U3 + CZ
brickwork ansatz (the n=26 recipe at a reduced size here; full size in
test_fullsize_gpu.py)."""
import numpy as np
import pytest

import oracle
from paper_2009_02823_gb300 import workloads as W
from tests.tolerances import TOL, grad_err

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("device", ["cpu", "cuda"])
@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_backward_matches_oracle(dtype, device):
    import torch

    from paper_2009_02823_gb300.autograd import VariationalEnergy
    w = W.config(5, n=11, layers=3)
    e_ref, g_ref = oracle.gradient_alg1(w.n, w.gates, w.theta, w.n_params, w.terms)
    m = VariationalEnergy(w.n, w.gates, w.n_params, w.terms, dtype, theta0=w.theta, device=device)
    e = m()
    e.backward()
    assert abs(float(e) - e_ref) <= TOL[dtype] * max(1.0, abs(e_ref))
    assert grad_err(m.theta.grad.cpu().numpy(), g_ref) <= TOL[dtype]
    # chain rule with an outer loss: d(3E^2)/dtheta = 6 E dE/dtheta
    m.theta.grad = None
    (3 * m() ** 2).backward()
    assert grad_err(m.theta.grad.cpu().numpy(), 6 * e_ref * g_ref) <= 10 * TOL[dtype]


def test_central_differences_subset():
    import torch

    from paper_2009_02823_gb300 import Circuit
    from paper_2009_02823_gb300.autograd import energy
    w = W.config(5, n=12, layers=2)
    c = Circuit(w.n, w.gates, w.n_params, "c128")
    c.set_hamiltonian(w.terms)
    th = torch.tensor(w.theta, requires_grad=True)
    energy(th, c).backward()
    rng = np.random.default_rng(5)
    d = 1e-4
    for p in rng.choice(w.n_params, 16, replace=False):
        tp, tm = w.theta.copy(), w.theta.copy()
        tp[p] += d
        tm[p] -= d
        fd = (c.energy(tp) - c.energy(tm)) / (2 * d)
        assert th.grad[p].item() == pytest.approx(fd, abs=1e-7)


def test_adam_descends():
    import torch

    from paper_2009_02823_gb300.autograd import VariationalEnergy
    w = W.config(5, n=12, layers=3)
    m = VariationalEnergy(w.n, w.gates, w.n_params, w.terms, "c64", theta0=w.theta, device="cuda")
    opt = torch.optim.Adam(m.parameters(), lr=0.01)
    first = None
    for _ in range(50):
        opt.zero_grad()
        e = m()
        e.backward()
        opt.step()
        first = float(e) if first is None else first
    last = float(m())
    assert np.isfinite(last) and last < first - 0.1
