"""``torch.autograd`` access to the library's adjoint gradient.

``EnergyFunction.apply(params, engine)`` returns the energy
<psi|H|psi>/<psi|psi> of the ansatz state for ``params`` (a float64 tensor
of ``engine.n_params`` values, on the host or the GPU).  When ``params``
requires a gradient, the forward runs the library's adjoint evaluation
(forward sweep, lambda = H psi, backward sweep) once and keeps the gradient
for ``backward``; otherwise it runs the energy evaluation alone.
"""
from __future__ import annotations

import torch

from .binding import Engine


def _energy_only(p: torch.Tensor, engine: Engine) -> torch.Tensor:
    if p.is_cuda:
        e = torch.empty(1, dtype=torch.float64, device=p.device)
        engine.energy_batch_dev(p.contiguous().view(1, -1), e)
        torch.cuda.current_stream(p.device).synchronize()
        return e[0]
    en, _ = engine.energy_batch(p.numpy().reshape(1, -1))
    return torch.tensor(float(en[0]), dtype=torch.float64)


def _energy_and_gradient(p: torch.Tensor, engine: Engine):
    if p.is_cuda:
        g = torch.empty(1, engine.n_params, dtype=torch.float64, device=p.device)
        e = torch.empty(1, dtype=torch.float64, device=p.device)
        engine.gradient_batch_dev(p.contiguous().view(1, -1), g, e)
        torch.cuda.current_stream(p.device).synchronize()
        return e[0], g.view(-1)
    gn, en = engine.gradient(p.numpy())
    return torch.tensor(en, dtype=torch.float64), torch.from_numpy(gn)


class EnergyFunction(torch.autograd.Function):
    @staticmethod
    def forward(ctx, params: torch.Tensor, engine: Engine):
        p = params.detach().to(dtype=torch.float64)
        if ctx.needs_input_grad[0]:
            energy, grad = _energy_and_gradient(p, engine)
            ctx.save_for_backward(grad)
        else:
            energy = _energy_only(p, engine)
        return energy.to(params.dtype)

    @staticmethod
    def backward(ctx, grad_out):
        (grad,) = ctx.saved_tensors
        return (grad_out * grad).to(grad_out.dtype), None


def energy_and_grad(params: torch.Tensor, engine: Engine) -> torch.Tensor:
    return EnergyFunction.apply(params, engine)
