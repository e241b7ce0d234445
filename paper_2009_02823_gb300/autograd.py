"""torch.autograd interface: the energy E(theta) of a variational circuit as a
differentiable function of theta, with the backward pass supplied by the library's
reverse-mode gradient (Algorithm 1).

    circ = Circuit(n, gates, P, "c64"); circ.set_hamiltonian(terms)
    theta = torch.tensor(theta0, dtype=torch.float64, requires_grad=True)
    E = energy(theta, circ)        # forward runs E and dE/dtheta in one library call
    E.backward()                   # theta.grad = dE/dtheta (chain rule with dL/dE)

theta may live on the CPU (host entry point, synchronous) or on the GPU (device entry
point on torch's current stream, no host synchronisation).  No CPU fallback exists:
the work always runs in libvqg.so.
"""
from __future__ import annotations

import torch

from .binding import Circuit


class _Energy(torch.autograd.Function):
    @staticmethod
    def forward(ctx, theta: torch.Tensor, circuit: Circuit):
        if theta.dim() != 1 or theta.numel() != circuit.n_params:
            raise ValueError(f"theta must be 1-D with {circuit.n_params} entries")
        th = theta.detach().to(torch.float64).contiguous()
        if th.is_cuda:
            stream = torch.cuda.current_stream(th.device)
            circuit.set_stream(stream)
            e = torch.empty(1, dtype=torch.float64, device=th.device)
            g = torch.empty(circuit.n_params, dtype=torch.float64, device=th.device)
            circuit.energy_and_gradient_device(th.data_ptr(), e.data_ptr(), g.data_ptr())
            e = e[0]
        else:
            ev, gv = circuit.energy_and_gradient(th.numpy())
            e = torch.tensor(ev, dtype=torch.float64)
            g = torch.from_numpy(gv.copy())
        ctx.save_for_backward(g)
        return e.to(theta.dtype)

    @staticmethod
    def backward(ctx, grad_e):
        (g,) = ctx.saved_tensors
        return (grad_e.to(g.dtype) * g).to(grad_e.dtype), None


def energy(theta: torch.Tensor, circuit: Circuit) -> torch.Tensor:
    """E(theta) with dE/dtheta from the reverse-mode sweep on backward()."""
    return _Energy.apply(theta, circuit)


class VariationalEnergy(torch.nn.Module):
    """A circuit + Hamiltonian as a module whose parameter is theta."""

    def __init__(self, n: int, gates, n_params: int, terms, dtype: str = "c64", theta0=None,
                 device: str | torch.device = "cpu", **circuit_options):
        super().__init__()
        self.circuit = Circuit(n, gates, n_params, dtype, **circuit_options)
        self.circuit.set_hamiltonian(terms)
        init = torch.zeros(n_params, dtype=torch.float64) if theta0 is None else \
            torch.as_tensor(theta0, dtype=torch.float64).clone()
        self.theta = torch.nn.Parameter(init.to(device))

    def forward(self) -> torch.Tensor:
        return energy(self.theta, self.circuit)
