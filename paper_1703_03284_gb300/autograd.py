"""torch.autograd.Function around the library's -2 ln L.

Forward calls ``mipwa_nll``; backward calls ``mipwa_nll_grad`` at the saved
parameters, so the per-event amplitudes are recomputed by the adjoint kernel
instead of being stored between the two passes.
"""
from __future__ import annotations

import torch


class MipwaNLL(torch.autograd.Function):
    """``MipwaNLL.apply(params, likelihood)`` -> 0-d float64 tensor (-2 ln L)."""

    @staticmethod
    def forward(ctx, params: torch.Tensor, likelihood):
        p = params.detach().to("cpu", torch.float64).contiguous()
        value = likelihood.nll(p.numpy())
        ctx.save_for_backward(params.detach())
        ctx.likelihood = likelihood
        return torch.tensor(value, dtype=torch.float64, device=params.device)

    @staticmethod
    def backward(ctx, grad_out: torch.Tensor):
        (params,) = ctx.saved_tensors
        p = params.to("cpu", torch.float64).contiguous()
        _, g = ctx.likelihood.nll_grad(p.numpy())
        g = torch.from_numpy(g).to(device=params.device, dtype=params.dtype)
        return grad_out.to(g.dtype) * g, None


def nll(params: torch.Tensor, likelihood) -> torch.Tensor:
    return MipwaNLL.apply(params, likelihood)
