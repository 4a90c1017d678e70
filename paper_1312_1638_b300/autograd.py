"""torch.autograd wrapper of the RK4 integrator and its discrete adjoint.

``FRStep.apply(u0, solver, dt, nsteps, every)`` returns u_N after `nsteps`
classical RK4 steps (fr_rk4); its backward pass runs fr_rk4_adjoint with
checkpoints every `every` steps.  Argument marshalling only: both passes run
in the library's kernels.  Single-block solvers (Euler or Navier-Stokes).
"""

from __future__ import annotations

import torch


class FRStep(torch.autograd.Function):
    @staticmethod
    def forward(ctx, u0, solver, dt, nsteps, every=10):
        if solver.nblocks != 1:
            raise ValueError("FRStep handles single-block meshes")
        u = u0.detach().clone().contiguous()
        solver.rk4([u], dt, nsteps)
        ctx.save_for_backward(u0.detach().contiguous())
        ctx.solver, ctx.dt, ctx.nsteps, ctx.every = solver, dt, nsteps, every
        return u

    @staticmethod
    def backward(ctx, grad):
        (u0,) = ctx.saved_tensors
        lam = grad.detach().clone().contiguous()
        ctx.solver.rk4_adjoint([u0], [lam], ctx.dt, ctx.nsteps, ctx.every)
        return lam, None, None, None, None
