"""``torch.autograd.Function`` wrappers of the library's adjoint kernels.

Argument marshalling only: the energy and its gradient are computed by
``mreg_warp_energy_grad`` in libmreg (see include/mreg.h); PyTorch supplies
the device tensors, the stream and the autograd graph.

    E = warp_energy(u, reg)      # E(u) = 1/2 sum_x (Te(x + u(x)) - Re(x))^2
    E.backward()                 # u.grad = dE/du  (n_nodes x 2)

    E = unrolled_warp_energy(u0, reg, 20)   # E(u_20), u_20 = 20 iterations from u0
    E.backward()                            # u0.grad = dE(u_20)/du0
"""
from __future__ import annotations

import torch

from . import mreg as _mreg

__all__ = ["WarpEnergy", "warp_energy", "UnrolledWarpEnergy", "unrolled_warp_energy"]


class WarpEnergy(torch.autograd.Function):
    """E(u) of a registration handle's images and mesh, FP64 scalar; its
    gradient with respect to u (FP32) is formed in the same call and kept
    for the backward pass."""

    @staticmethod
    def forward(ctx, u: torch.Tensor, reg: "_mreg.Registration") -> torch.Tensor:
        uc = u.detach().to(torch.float32).contiguous()
        energy = torch.empty(1, dtype=torch.float64, device=u.device)
        grad = torch.empty_like(uc) if ctx.needs_input_grad[0] else None
        reg.warp_energy_grad(uc, energy, grad)
        ctx.save_for_backward(grad)
        return energy.reshape(())

    @staticmethod
    def backward(ctx, g_energy: torch.Tensor):
        (grad,) = ctx.saved_tensors
        if grad is None:
            return None, None
        return (grad * g_energy.to(grad.dtype)), None


def warp_energy(u: torch.Tensor, reg: "_mreg.Registration") -> torch.Tensor:
    return WarpEnergy.apply(u, reg)


class UnrolledWarpEnergy(torch.autograd.Function):
    """E(u_K) with u_K = K explicit iterations (spline gradient) of the
    handle's loop from u0; its gradient with respect to u0 comes from the
    library's adjoint recursion over the kept states."""

    @staticmethod
    def forward(ctx, u0: torch.Tensor, reg: "_mreg.Registration", n_iters: int,
                checkpoint_every: int = 0) -> torch.Tensor:
        uc = u0.detach().to(torch.float32).contiguous()
        energy = torch.empty(1, dtype=torch.float64, device=u0.device)
        grad = torch.empty_like(uc) if ctx.needs_input_grad[0] else None
        reg.unroll_grad(uc, n_iters, energy, grad, checkpoint_every=checkpoint_every)
        ctx.save_for_backward(grad)
        ctx.reg = reg
        return energy.reshape(())

    @staticmethod
    def backward(ctx, g_energy: torch.Tensor):
        (grad,) = ctx.saved_tensors
        if grad is None:
            return None, None, None, None
        # the forward run is a persistent kernel with bounded grid-barrier
        # waits: raise (MregError, MREG_ERR_DEVICE_CHECK) if one gave up
        # rather than hand back a gradient of an unfinished run
        ctx.reg.stats()
        return (grad * g_energy.to(grad.dtype)), None, None, None


def unrolled_warp_energy(u0: torch.Tensor, reg: "_mreg.Registration", n_iters: int,
                         checkpoint_every: int = 0) -> torch.Tensor:
    """E(u_K) with its gradient through the K iterations; checkpoint_every
    > 0 keeps only every c-th state of the forward run and recomputes the
    segments in the backward pass (the same gradient, bit for bit)."""
    return UnrolledWarpEnergy.apply(u0, reg, n_iters, checkpoint_every)
