"""torch.autograd bindings of the explicit and BTCS solves.

``burgers_solve(ctx, scheme, batch, u0, nu)`` returns u(T) for every row of
the packed batch; its backward runs the library's hand-written adjoint kernels
(reverse stencil / transposed cyclic solve, sqrt-step checkpointing, FP64
viscosity accumulators) and yields dJ/du0 and dJ/dnu. dt, dx and the step
counts are held fixed (they are taken from the batch, not differentiated).
"""
from __future__ import annotations

import numpy as np
import torch

from .api import Batch, Context


class BurgersSolve(torch.autograd.Function):
    @staticmethod
    def forward(fctx, u0: torch.Tensor, nu: torch.Tensor, lib: Context, scheme: int,
                batch: Batch, ckpt_stride: int):
        nus = nu.detach().to("cpu", torch.float64).numpy()
        b = batch.with_fields(nu=nus)
        u = u0.detach().clone().contiguous()
        lib.advance(scheme, b, u)
        fctx.save_for_backward(u0.detach())
        fctx.lib, fctx.scheme, fctx.batch, fctx.stride = lib, scheme, b, ckpt_stride
        fctx.nu_meta = (nu.dtype, nu.device)
        return u

    @staticmethod
    def backward(fctx, gout: torch.Tensor):
        (u0,) = fctx.saved_tensors
        g = gout.contiguous()
        if g.dtype != u0.dtype:
            g = g.to(u0.dtype)
        gu0 = torch.zeros_like(u0)
        gnu = torch.empty(fctx.batch.count, dtype=torch.float64, device=u0.device)
        fctx.lib.adjoint(fctx.scheme, fctx.batch, u0, g, gu0, gnu, fctx.stride)
        dtype, device = fctx.nu_meta
        return gu0, gnu.to(device=device, dtype=dtype), None, None, None, None


def burgers_solve(lib: Context, scheme: int, batch: Batch, u0: torch.Tensor, nu: torch.Tensor,
                  ckpt_stride: int = 0) -> torch.Tensor:
    """Differentiable packed-batch solve: u(T) = solve(u0; nu)."""
    if nu.numel() != batch.count:
        raise ValueError("nu needs one value per row")
    return BurgersSolve.apply(u0, nu, lib, scheme, batch, int(ckpt_stride))


def misfit_loss(uT: torch.Tensor, target: torch.Tensor) -> torch.Tensor:
    """J = 1/2 sum (u(T) - target)^2 accumulated in FP64."""
    d = (uT - target).double()
    return 0.5 * torch.sum(d * d)


__all__ = ["BurgersSolve", "burgers_solve", "misfit_loss", "np"]
