"""torch.autograd.Function over the forward run and its adjoint.

`seismograms(sim, lam, mu, rho, nt, dt)` returns the [3][nrec][nt]
seismograms of the simulation for the medium (lam, mu, rho) given as CUDA
tensors; backpropagating through it calls ews_adjoint, which re-runs the
forward loop with checkpoints and steps the exact discrete adjoint back.
All numerical work is in libews; this module only passes pointers.
"""
from __future__ import annotations

import torch

from . import ews


class _ElasticSeismograms(torch.autograd.Function):
    @staticmethod
    def forward(ctx, lam, mu, rho, sim, nt, dt, ckpt_every):
        for t in (lam, mu, rho):
            if not (t.is_cuda and t.dtype == torch.float32):
                raise TypeError("lam, mu, rho must be float32 CUDA tensors")
        lam, mu, rho = lam.contiguous(), mu.contiguous(), rho.contiguous()
        sim.set_stream(torch.cuda.current_stream().cuda_stream)
        sim.set_model_lame(lam, mu, rho)
        seis = torch.zeros((3, sim.nrec, nt), device=lam.device, dtype=torch.float32)
        sim.run(nt, dt, seis if sim.nrec else None)
        ctx.save_for_backward(lam, mu, rho)
        ctx.sim, ctx.nt, ctx.dt, ctx.ckpt = sim, nt, dt, ckpt_every
        return seis

    @staticmethod
    def backward(ctx, grad_seis):
        lam, mu, rho = ctx.saved_tensors
        sim = ctx.sim
        sim.set_stream(torch.cuda.current_stream().cuda_stream)
        sim.set_model_lame(lam, mu, rho)           # the model the forward saw
        g = torch.empty((3,) + tuple(lam.shape), device=lam.device, dtype=torch.float32)
        ews.ews_adjoint(sim.handle, ctx.nt, ctx.dt, grad_seis.contiguous().float(), g[0], g[1],
                        g[2], ctx.ckpt)
        return g[0], g[1], g[2], None, None, None, None


def seismograms(sim: ews.Simulation, lam: torch.Tensor, mu: torch.Tensor, rho: torch.Tensor,
                nt: int, dt: float, ckpt_every: int = 0) -> torch.Tensor:
    """Differentiable forward run: seismograms [3][nrec][nt] of `sim` (source
    and receivers already set) for the medium (lam, mu, rho)."""
    return _ElasticSeismograms.apply(lam, mu, rho, sim, int(nt), float(dt), int(ckpt_every))
