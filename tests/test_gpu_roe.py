"""Roe flux on the GPU (CPR and FV schemes) against the FP64 oracle through
the C ABI.  Tolerances as for the Rusanov runs: FP64 <= 1e-12, FP32 <= 1e-5
relative L2."""
import numpy as np
import pytest
import torch

import oracle
from paper_1709_01619_gb300 import _native as nat
from paper_1709_01619_gb300 import inputs

pytestmark = pytest.mark.gpu

TOL64, TOL32 = 1e-12, 1e-5


def make(dtype=nat.F64, **kw):
    kw.setdefault("flux", nat.ROE)
    c = nat.Config(dtype=dtype, **kw)
    o = oracle.Config(eqn=c.eqn, nx=c.nx, ny=c.ny, p=c.p, x0=c.x0, x1=c.x1, y0=c.y0, y1=c.y1,
                      pts=c.pts, div=c.div, flux=oracle.ROE, ax=c.ax, ay=c.ay, gamma=c.gamma,
                      bc_x=c.bc_x, bc_y=c.bc_y, limiter=c.limiter, tvb_M=c.tvb_M, lim_eps=c.lim_eps,
                      cfl=c.cfl, scheme=c.scheme)
    return c, o


def rel(a, b):
    a, b = np.asarray(a, np.float64).ravel(), np.asarray(b, np.float64).ravel()
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def dev(q, c):
    return torch.tensor(np.asarray(q).reshape(c.shape), dtype=c.torch_dtype, device="cuda")


def host(t):
    return t.detach().double().cpu().numpy()


CASES = [dict(p=p, pts=pts, div=div, bc=bc) for p in (1, 2, 3, 4) for pts in (0, 1) for div in (0, 1)
         for bc in (0, 1) if (p + pts + div + bc) % 2 == 0]


@pytest.mark.parametrize("case", CASES, ids=lambda c: "-".join(f"{k}{v}" for k, v in c.items()))
@pytest.mark.parametrize("dtype", [nat.F64, nat.F32])
def test_cpr_residual_parity(case, dtype):
    c, o = make(dtype, eqn=nat.EULER, nx=19, ny=13, p=case["p"], pts=case["pts"], div=case["div"],
                bc_x=case["bc"], bc_y=case["bc"], x1=4.0, y1=3.0)
    x, y = oracle.point_coords(o)
    # smooth data: the edge states interpolated from a discontinuous field can
    # leave the physical range, where no flux is defined
    q = inputs.perturbed(inputs.vortex(x, y, eps=3.0, xc=2.0, yc=1.5, lx=4.0, ly=3.0), 11, 0.02)
    if dtype == nat.F32:
        q = q.astype(np.float32).astype(np.float64)
    R_or = oracle.residual(o, q)
    with nat.Context(c) as ctx:
        R = host(ctx.residual(dev(q, c)))
    assert rel(R, R_or) <= (TOL64 if dtype == nat.F64 else TOL32)


@pytest.mark.parametrize("dtype", [nat.F64, nat.F32])
def test_fv_residual_parity(dtype):
    c, o = make(dtype, eqn=nat.EULER, nx=45, ny=21, p=0, scheme=nat.SCHEME_FV_MUSCL,
                bc_x=nat.TRANSMISSIVE, bc_y=nat.TRANSMISSIVE)
    x, y = oracle.point_coords(o)
    q = inputs.perturbed(inputs.four_quadrant(x, y), 5, 0.02)
    if dtype == nat.F32:
        q = q.astype(np.float32).astype(np.float64)
    R_or = oracle.residual(o, q)
    with nat.Context(c) as ctx:
        R = host(ctx.residual(dev(q, c)))
    assert rel(R, R_or) <= (TOL64 if dtype == nat.F64 else TOL32)


def test_limited_steps_fp64():
    c, o = make(nat.F64, eqn=nat.EULER, nx=40, ny=40, p=2, bc_x=nat.TRANSMISSIVE, bc_y=nat.TRANSMISSIVE,
                limiter=1, tvb_M=50.0, lim_eps=1e-3, cfl=0.1)
    x, y = oracle.point_coords(o)
    q0, _, _, _ = oracle.limit(o, inputs.four_quadrant(x, y))
    q_or, _, _ = oracle.run(o, q0, 6, 2e-4)
    with nat.Context(c) as ctx:
        qd = dev(q0, c)
        ctx.step(qd, 6, 2e-4)
        q = host(qd)
    assert rel(q, q_or) <= TOL64


def test_fp32_cfl_run_to_t_end():
    c, o = make(nat.F32, eqn=nat.EULER, nx=24, ny=20, p=3, x1=10.0, y1=10.0, cfl=0.08)
    x, y = oracle.point_coords(o)
    q0 = inputs.vortex(x, y, eps=5.0).astype(np.float32).astype(np.float64)
    q_or, n_or, _ = oracle.run(o, q0, 10000, 0.0, 0.2)
    with nat.Context(c) as ctx:
        qd = dev(q0, c)
        ctx.step(qd, n_or + 3, 0.0, 0.2)
        t, n = ctx.get_time()
        q = host(qd)
    assert t == 0.2 and n == n_or
    assert rel(q, q_or) <= 1e-6


def test_roe_has_no_adjoint():
    c, _ = make(nat.F64, eqn=nat.EULER, nx=8, ny=8, p=2)
    with nat.Context(c) as ctx:
        q = torch.ones(c.shape, dtype=torch.float64, device="cuda")
        with pytest.raises(nat.CprError):
            ctx.residual_vjp(q, q)
