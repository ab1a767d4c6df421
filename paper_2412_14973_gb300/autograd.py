"""torch.autograd.Function over the library's misfit and factor gradients.

``TLRMisfit.apply(theta, handle)`` returns f = 0.5 ||D-hat C(theta) - U-hat||^2
(eq. 17a) as a real scalar tensor; its backward returns grad_out times the
factor gradients of eq. (25)-(27), which the library computes in one call.
For a real function of complex inputs PyTorch propagates
dL/dRe(z) + i dL/dIm(z), which is the convention of eq. (25)-(27), so the
library's gradient is passed through unchanged.  Marshalling only: both
directions run in the CUDA library.
"""
from __future__ import annotations

import torch

from . import tlr_mdd as T


class TLRMisfit(torch.autograd.Function):
    @staticmethod
    def forward(ctx, theta: torch.Tensor, handle: int):
        if theta.dtype != torch.complex64 or not theta.is_cuda:
            raise TypeError("theta must be a complex64 CUDA tensor")
        th = theta.detach().contiguous()
        g = torch.empty_like(th)
        f = T.tlr_mdd_grad(handle, th, g, want_f=True)
        ctx.save_for_backward(g)
        return torch.tensor(f, dtype=torch.float64, device=theta.device)

    @staticmethod
    def backward(ctx, grad_out):
        (g,) = ctx.saved_tensors
        return (grad_out.to(torch.float32) * g, None)


def misfit(theta: torch.Tensor, handle: int) -> torch.Tensor:
    """Differentiable f(theta) for one handle (one frequency)."""
    return TLRMisfit.apply(theta, handle)
