"""torch.autograd wrapper of the adjoint: the trace misfit of a shot as a
differentiable function of the velocity model."""
from __future__ import annotations

import torch

from . import seisgb


class VelocityMisfit(torch.autograd.Function):
    """J(v) = 1/2 sum_{n,r} (d^n_r(v) - observed^n_r)^2 for one shot.

    forward(velocity, grid, wavelet, nt, src_ijk, rec_ijk, observed, ckpt_every)
    returns J as a 0-d float64 tensor; backward gives grad_output * dJ/dv from the
    hand-written adjoint (computed in forward, fp64 time accumulation), cast to
    the velocity's dtype.  velocity: CUDA float32 tensor (Nz, Ny, Nx)."""

    @staticmethod
    def forward(ctx, velocity, grid, wavelet, nt, src_ijk, rec_ijk, observed, ckpt_every=0):
        v = velocity.detach().contiguous()
        grad = torch.empty(v.shape, dtype=torch.float64, device=v.device)
        J = seisgb.adjoint_shot(grid, v, wavelet.contiguous(), nt, src_ijk, rec_ijk,
                                observed.contiguous(), grad, ckpt_every)
        ctx.save_for_backward(grad)
        ctx.vdtype = velocity.dtype
        return torch.tensor(J, dtype=torch.float64, device=v.device)

    @staticmethod
    def backward(ctx, grad_output):
        (grad,) = ctx.saved_tensors
        return (grad_output * grad).to(ctx.vdtype), None, None, None, None, None, None, None


def velocity_misfit(velocity, grid, wavelet, nt, src_ijk, rec_ijk, observed, ckpt_every=0):
    return VelocityMisfit.apply(velocity, grid, wavelet, nt, src_ijk, rec_ijk, observed, ckpt_every)
