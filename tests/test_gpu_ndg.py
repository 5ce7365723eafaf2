"""Nodal-DG edge correction (Sec. 2.3) on the GPU against the FP64 oracle,
through the C ABI: the lift of the strong form with the exact mass matrix
(CPR_CORR_NDG, the same scheme as the Radau correction) and with the lumped
one (CPR_CORR_NDG_LUMPED, a different scheme on Gauss-Lobatto points).

Tolerances as for the other parity tests: FP64 <= 1e-12 relative L2, FP32
<= 1e-5 for a residual and <= 1e-6 after fixed steps."""
import numpy as np
import pytest
import torch

import oracle
from paper_1709_01619_gb300 import _native as nat
from paper_1709_01619_gb300 import inputs

pytestmark = pytest.mark.gpu

TOL64, TOL32 = 1e-12, 1e-5
CORRS = [nat.CORR_NDG, nat.CORR_NDG_LUMPED]


def make(dtype=nat.F64, **kw):
    c = nat.Config(dtype=dtype, **kw)
    o = oracle.Config(eqn=c.eqn, nx=c.nx, ny=c.ny, p=c.p, x0=c.x0, x1=c.x1, y0=c.y0, y1=c.y1,
                      pts=c.pts, div=c.div, flux=c.flux, ax=c.ax, ay=c.ay, gamma=c.gamma,
                      bc_x=c.bc_x, bc_y=c.bc_y, cfl=c.cfl, corr=c.corr)
    return c, o


def rel(a, b):
    a, b = np.asarray(a, np.float64).ravel(), np.asarray(b, np.float64).ravel()
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def dev(q, c):
    return torch.tensor(np.asarray(q).reshape(c.shape), dtype=c.torch_dtype, device="cuda")


def host(t):
    return t.detach().double().cpu().numpy()


def vortex_state(o, seed):
    x, y = oracle.point_coords(o)
    q = inputs.vortex(x, y, eps=3.0, xc=0.5 * o.x1, yc=0.5 * o.y1, lx=o.x1, ly=o.y1)
    return inputs.perturbed(q, seed, 0.02)


@pytest.mark.parametrize("corr", CORRS)
@pytest.mark.parametrize("pts", [nat.GAUSS, nat.LOBATTO])
@pytest.mark.parametrize("p", [1, 2, 3, 4])
@pytest.mark.parametrize("dtype", [nat.F64, nat.F32])
def test_euler_residual_parity(corr, pts, p, dtype):
    c, o = make(dtype, eqn=nat.EULER, nx=19, ny=11, p=p, pts=pts, corr=corr, x1=4.0, y1=2.5,
                bc_x=nat.TRANSMISSIVE if p % 2 else nat.PERIODIC)
    q = vortex_state(o, p)
    if dtype == nat.F32:
        q = q.astype(np.float32).astype(np.float64)
    R_or = oracle.residual(o, q)
    with nat.Context(c) as ctx:
        R = host(ctx.residual(dev(q, c)))
    assert rel(R, R_or) <= (TOL64 if dtype == nat.F64 else TOL32)


@pytest.mark.parametrize("corr", CORRS)
def test_advection_residual_parity(corr):
    c, o = make(nat.F64, eqn=nat.ADVECTION, nx=21, ny=10, p=3, pts=nat.LOBATTO, corr=corr,
                flux=nat.UPWIND, ax=0.8, ay=-0.5)
    q = np.random.default_rng(3).standard_normal(c.shape)
    R_or = oracle.residual(o, q)
    with nat.Context(c) as ctx:
        R = host(ctx.residual(dev(q, c)))
    assert rel(R, R_or) <= TOL64


@pytest.mark.parametrize("dtype", [nat.F64, nat.F32])
def test_lumped_lobatto_fixed_steps(dtype):
    c, o = make(dtype, eqn=nat.EULER, nx=24, ny=18, p=3, pts=nat.LOBATTO, corr=nat.CORR_NDG_LUMPED,
                x1=8.0, y1=6.0)
    q0 = vortex_state(o, 9)
    if dtype == nat.F32:
        q0 = q0.astype(np.float32).astype(np.float64)
    q_or, _, _ = oracle.run(o, q0, 5, 2e-3)
    with nat.Context(c) as ctx:
        qd = dev(q0, c)
        ctx.step(qd, 5, 2e-3)
        q = host(qd)
    assert rel(q, q_or) <= (TOL64 if dtype == nat.F64 else 1e-6)


def test_lumped_lobatto_cfl_run_lands_on_t_end():
    c, o = make(nat.F64, eqn=nat.EULER, nx=20, ny=20, p=2, pts=nat.LOBATTO, corr=nat.CORR_NDG_LUMPED,
                x1=10.0, y1=10.0, cfl=0.1)
    x, y = oracle.point_coords(o)
    q0 = inputs.vortex(x, y, eps=5.0)
    q_or, n_or, t_or = oracle.run(o, q0, 10000, 0.0, 0.15)
    with nat.Context(c) as ctx:
        qd = dev(q0, c)
        ctx.step(qd, n_or + 3, 0.0, 0.15)
        t, n = ctx.get_time()
        q = host(qd)
    assert n == n_or and t == t_or == 0.15
    assert rel(q, q_or) <= TOL64


def test_lumped_lobatto_residual_vjp():
    c, o = make(nat.F64, eqn=nat.EULER, nx=9, ny=8, p=3, pts=nat.LOBATTO, corr=nat.CORR_NDG_LUMPED,
                x1=4.5, y1=4.0)
    q = vortex_state(o, 4)
    rbar = np.random.default_rng(2).standard_normal(c.shape)
    qb_or = oracle.residual_vjp(o, q, rbar)
    with nat.Context(c) as ctx:
        qb = host(ctx.residual_vjp(dev(q, c), dev(rbar, c)))
    assert rel(qb, qb_or) <= TOL64
