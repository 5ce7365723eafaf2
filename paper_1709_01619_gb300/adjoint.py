"""Gradients through many SSP-RK3 steps: torch.autograd.Function over the
hand-written discrete adjoint (cpr_step_vjp), with checkpointed recomputation.

The forward pass advances q0 by ``nsteps`` fixed steps of size ``dt`` and keeps
the state every ``every`` steps.  The backward pass walks the segments in
reverse: it recomputes the states of one segment from its checkpoint and
applies the transposed step to the cotangent, last step first.  Memory: one
state per checkpoint plus one segment of states.  Valid for unlimited runs
with the LP divergence (the adjoint of the limiter is not defined).
"""
from __future__ import annotations

import torch

from ._native import Context


class CPRRollout(torch.autograd.Function):
    @staticmethod
    def forward(ctx, q0, solver: Context, nsteps: int, dt: float, every: int):
        q = q0.detach().contiguous().clone()
        ckpts = []
        for s in range(nsteps):
            if s % every == 0:
                ckpts.append(q.clone())
            solver.step(q, 1, dt)
        ctx.solver, ctx.nsteps, ctx.dt, ctx.every, ctx.ckpts = solver, nsteps, dt, every, ckpts
        return q

    @staticmethod
    def backward(ctx, gout):
        solver, nsteps, dt, every = ctx.solver, ctx.nsteps, ctx.dt, ctx.every
        qbar = gout.contiguous().clone()
        tmp = torch.empty_like(qbar)
        for k in reversed(range(len(ctx.ckpts))):
            start = k * every
            end = min(start + every, nsteps)
            states = [ctx.ckpts[k]]
            q = ctx.ckpts[k].clone()
            for _ in range(start, end - 1):
                solver.step(q, 1, dt)
                states.append(q.clone())
            for s in reversed(range(end - start)):
                solver.step_vjp(states[s], qbar, dt, tmp)
                qbar, tmp = tmp, qbar
        return qbar, None, None, None, None


def rollout(q0, solver: Context, nsteps: int, dt: float, every: int = 20):
    """q after ``nsteps`` SSP-RK3 steps of size ``dt`` from ``q0``,
    differentiable with respect to ``q0``."""
    if nsteps < 1 or every < 1:
        raise ValueError("nsteps and every must be >= 1")
    return CPRRollout.apply(q0, solver, int(nsteps), float(dt), int(every))


def quadrature_weights(solver: Context) -> torch.Tensor:
    """(hx hy / 4) w_a w_b at every solution point, broadcast over variables:
    the weights of the L2 misfit J = 1/2 sum W (q - q_target)^2."""
    import numpy as np
    c = solver.cfg
    n = c.p + 1
    x, y = solver.point_coords()
    hx, hy = (c.x1 - c.x0) / c.nx, (c.y1 - c.y0) / c.ny
    # quadrature weights from the points of one element: the Gauss rule of
    # the reference interval, recovered from numpy's Legendre module
    xi, w = np.polynomial.legendre.leggauss(n)
    W2 = (hx * hy / 4.0) * np.outer(w, w).reshape(n * n)  # [b, a]
    W = np.broadcast_to(W2, (c.nvars, c.ne, n * n))
    return torch.tensor(np.ascontiguousarray(W), dtype=c.torch_dtype, device="cuda")
