"""Gradients through many SSP-RK3 steps: torch.autograd.Function over the
hand-written discrete adjoint (cpr_step_stages, cpr_step_vjp_stages), with
checkpointed recomputation.

The forward pass advances q0 by ``nsteps`` fixed steps of size ``dt`` and keeps
the state every ``every`` steps.  The backward pass walks the segments in
reverse: it recomputes the states of one segment from its checkpoint, with the
stage states of each step (the Shu-Osher form of Sec. 4), and applies the
transposed step around them to the cotangent, last step first.  Memory: one
state per checkpoint plus three states per step of one segment.  Valid for
unlimited runs with the LP divergence (the adjoint of the limiter is not
defined).
"""
from __future__ import annotations

import torch

from ._native import Context


class CPRRollout(torch.autograd.Function):
    @staticmethod
    def forward(ctx, q0, solver: Context, nsteps: int, dt: float, every: int):
        q = q0.detach().contiguous().clone()
        ckpts = []
        for s in range(0, nsteps, every):
            ckpts.append(q.clone())
            # a segment in one call: the step graphs run back to back
            solver.step(q, min(every, nsteps - s), dt)
        ctx.solver, ctx.nsteps, ctx.dt, ctx.every, ctx.ckpts = solver, nsteps, dt, every, ckpts
        return q

    @staticmethod
    def backward(ctx, gout):
        solver, nsteps, dt, every = ctx.solver, ctx.nsteps, ctx.dt, ctx.every
        qbar = gout.contiguous().clone()
        tmp = torch.empty_like(qbar)
        # Buffers for one segment, allocated once per backward pass: its
        # states after the checkpoint and the two stage states of each of its
        # steps, so that the reverse sweep applies only the three transposed
        # residuals per step (cpr_step_vjp_stages) instead of recomputing the
        # stages.
        n = min(every, nsteps)
        xs = [torch.empty_like(qbar) for _ in range(n)]
        s1 = [torch.empty_like(qbar) for _ in range(n)]
        s2 = [torch.empty_like(qbar) for _ in range(n)]
        for k in reversed(range(len(ctx.ckpts))):
            start = k * every
            m = min(start + every, nsteps) - start
            states = [ctx.ckpts[k]]
            for s in range(m):
                solver.step_stages(states[s], s1[s], s2[s], xs[s], dt)
                states.append(xs[s])
            for s in reversed(range(m)):
                solver.step_vjp_stages(states[s], s1[s], s2[s], qbar, dt, tmp)
                qbar, tmp = tmp, qbar
        return qbar, None, None, None, None


def rollout(q0, solver: Context, nsteps: int, dt: float, every: int = 20):
    """q after ``nsteps`` SSP-RK3 steps of size ``dt`` from ``q0``,
    differentiable with respect to ``q0``."""
    if nsteps < 1 or every < 1:
        raise ValueError("nsteps and every must be >= 1")
    return CPRRollout.apply(q0, solver, int(nsteps), float(dt), int(every))


def point_weights(n: int, lobatto: bool):
    """Quadrature weights of the n solution points on [-1, 1]: the Gauss rule,
    or the Gauss-Lobatto rule 2 / (n (n - 1) P_{n-1}(x)^2) at its nodes (the
    ends and the roots of P'_{n-1}), from numpy's Legendre module."""
    import numpy as np
    if not lobatto or n < 2:
        return np.polynomial.legendre.leggauss(n)[1]
    pn1 = np.polynomial.legendre.Legendre.basis(n - 1)
    xi = np.concatenate(([-1.0], np.sort(pn1.deriv().roots().real), [1.0]))
    return 2.0 / (n * (n - 1) * pn1(xi) ** 2)


def quadrature_weights(solver: Context) -> torch.Tensor:
    """(hx hy / 4) w_a w_b at every solution point, broadcast over variables:
    the weights of the L2 misfit J = 1/2 sum W (q - q_target)^2, w the
    quadrature weights of the configuration's solution points."""
    import numpy as np
    from ._native import LOBATTO
    c = solver.cfg
    n = c.p + 1
    hx, hy = (c.x1 - c.x0) / c.nx, (c.y1 - c.y0) / c.ny
    w = point_weights(n, c.pts == LOBATTO)
    W2 = (hx * hy / 4.0) * np.outer(w, w).reshape(n * n)  # [b, a]
    W = np.broadcast_to(W2, (c.nvars, c.ne, n * n))
    return torch.tensor(np.ascontiguousarray(W), dtype=c.torch_dtype,
                        device="cuda" if torch.cuda.is_available() else "cpu")
