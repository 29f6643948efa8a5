"""``torch.autograd`` access to the library's adjoint gradient.

``EnergyFunction.apply(params, engine)`` returns the energy
<psi|H|psi>/<psi|psi> of the ansatz state for ``params`` (a float64 tensor
of ``engine.n_params`` values, on the host or the GPU) and, on backward,
the gradient from the library's adjoint sweep (``vqe_gradient``).
"""
from __future__ import annotations

import torch

from .binding import Engine


class EnergyFunction(torch.autograd.Function):
    @staticmethod
    def forward(ctx, params: torch.Tensor, engine: Engine):
        p = params.detach().to(dtype=torch.float64)
        if p.is_cuda:
            g = torch.empty(1, engine.n_params, dtype=torch.float64, device=p.device)
            e = torch.empty(1, dtype=torch.float64, device=p.device)
            engine.gradient_batch_dev(p.contiguous().view(1, -1), g, e)
            torch.cuda.current_stream(p.device).synchronize()
            grad = g.view(-1)
            energy = e[0]
        else:
            gn, en = engine.gradient(p.numpy())
            grad = torch.from_numpy(gn)
            energy = torch.tensor(en, dtype=torch.float64)
        ctx.save_for_backward(grad)
        return energy.to(params.dtype)

    @staticmethod
    def backward(ctx, grad_out):
        (grad,) = ctx.saved_tensors
        return (grad_out * grad).to(grad_out.dtype), None


def energy_and_grad(params: torch.Tensor, engine: Engine) -> torch.Tensor:
    return EnergyFunction.apply(params, engine)
