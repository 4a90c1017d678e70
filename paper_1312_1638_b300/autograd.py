"""torch.autograd wrappers of the RK4 integrator and its discrete adjoint.

``FRStep.apply(u0, solver, dt, nsteps, every)`` returns u_N after `nsteps`
classical RK4 steps (fr_rk4) of a single-block solver; its backward pass runs
fr_rk4_adjoint with checkpoints every `every` steps.

``FRStepBlocks.apply(solver, dt, nsteps, every, *u0)`` does the same for a
solver with any number of element blocks (a mixed mesh: one state tensor per
block, in the solver's block order) and returns a tuple of per-block states;
``rk4(solver, u0, dt, nsteps, every)`` picks the right one for a tensor or a
sequence of tensors.  Argument marshalling only: both passes run in the
library's kernels.
"""

from __future__ import annotations

import torch


class FRStep(torch.autograd.Function):
    @staticmethod
    def forward(ctx, u0, solver, dt, nsteps, every=10):
        if solver.nblocks != 1:
            raise ValueError("FRStep handles single-block meshes; use FRStepBlocks")
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


class FRStepBlocks(torch.autograd.Function):
    @staticmethod
    def forward(ctx, solver, dt, nsteps, every, *u0):
        if len(u0) != solver.nblocks:
            raise ValueError(f"expected {solver.nblocks} block states, got {len(u0)}")
        u = [x.detach().clone().contiguous() for x in u0]
        solver.rk4(u, dt, nsteps)
        ctx.save_for_backward(*[x.detach().contiguous() for x in u0])
        ctx.solver, ctx.dt, ctx.nsteps, ctx.every = solver, dt, nsteps, every
        return tuple(u)

    @staticmethod
    def backward(ctx, *grads):
        u0 = list(ctx.saved_tensors)
        # a block whose output does not reach the loss contributes a zero cotangent
        lam = [torch.zeros_like(x) if g is None else g.detach().clone().contiguous() for g, x in zip(grads, u0)]
        ctx.solver.rk4_adjoint(u0, lam, ctx.dt, ctx.nsteps, ctx.every)
        return (None, None, None, None, *lam)


def rk4(solver, u0, dt, nsteps, every=10):
    """u_N = RK4^nsteps(u0), differentiable: u0 is one tensor (single block)
    or a sequence of per-block tensors (returns a tuple then)."""
    if isinstance(u0, torch.Tensor):
        return FRStep.apply(u0, solver, dt, nsteps, every)
    return FRStepBlocks.apply(solver, dt, nsteps, every, *u0)
