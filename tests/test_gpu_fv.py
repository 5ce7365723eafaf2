"""FV MUSCL-minmod schemes (Sec. 2.1, 2.6, Algorithm 1; second- and
third-order reconstruction) on the GPU against the FP64 oracle, through the
C ABI: residual, fixed and CFL steps, the
conservation of the averages, and the four-quadrant problem of the equal-DOF
comparison at full size (1536 x 1536 elements).

Tolerances: FP64 <= 1e-12 relative L2 (rounding order only), FP32 <= 1e-5;
FP32 fixed steps <= 1e-6 (as for CPR).  Grids span several 32 x 8 element
tiles with ragged tails."""
import numpy as np
import pytest
import torch

import oracle
from paper_1709_01619_gb300 import _native as nat
from paper_1709_01619_gb300 import inputs

pytestmark = pytest.mark.gpu

TOL64, TOL32 = 1e-12, 1e-5


ORDERS = [nat.SCHEME_FV_MUSCL, nat.SCHEME_FV_MUSCL3]
TO_ORACLE = {nat.SCHEME_FV_MUSCL: oracle.FV_MUSCL, nat.SCHEME_FV_MUSCL3: oracle.FV_MUSCL3}


def make(dtype=nat.F64, **kw):
    kw.setdefault("p", 0)
    kw.setdefault("scheme", nat.SCHEME_FV_MUSCL)
    c = nat.Config(dtype=dtype, **kw)
    o = oracle.Config(eqn=c.eqn, nx=c.nx, ny=c.ny, p=0, x0=c.x0, x1=c.x1, y0=c.y0, y1=c.y1,
                      flux=c.flux, ax=c.ax, ay=c.ay, gamma=c.gamma, bc_x=c.bc_x, bc_y=c.bc_y,
                      cfl=c.cfl, scheme=TO_ORACLE[c.scheme])
    return c, o


def rel(a, b):
    a, b = np.asarray(a, np.float64).ravel(), np.asarray(b, np.float64).ravel()
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def dev(q, c):
    return torch.tensor(np.asarray(q).reshape(c.shape), dtype=c.torch_dtype, device="cuda")


def host(t):
    return t.detach().double().cpu().numpy()


def state(o, kind, seed):
    x, y = oracle.point_coords(o)
    if o.eqn == oracle.ADVECTION:
        return np.random.default_rng(seed).standard_normal((1, o.ne, 1))
    if kind == "vortex":
        q = inputs.vortex(x, y, eps=3.0, xc=0.5 * o.x1, yc=0.5 * o.y1, lx=o.x1, ly=o.y1)
    else:
        q = inputs.four_quadrant(x, y)
    return inputs.perturbed(q, seed, 0.02)


CASES = [
    dict(eqn=nat.EULER, nx=37, ny=29, x1=3.0, y1=2.0, kind="vortex"),
    dict(eqn=nat.EULER, nx=70, ny=9, bc_x=nat.TRANSMISSIVE, bc_y=nat.TRANSMISSIVE, kind="4q"),
    dict(eqn=nat.EULER, nx=33, ny=17, bc_x=nat.TRANSMISSIVE, kind="vortex"),
    dict(eqn=nat.EULER, nx=1, ny=5, kind="vortex"),
    dict(eqn=nat.EULER, nx=2, ny=3, bc_y=nat.TRANSMISSIVE, kind="4q"),
    dict(eqn=nat.ADVECTION, nx=45, ny=13, flux=nat.UPWIND, ax=0.7, ay=-1.2, kind=""),
    dict(eqn=nat.ADVECTION, nx=31, ny=40, flux=nat.RUSANOV, ax=-0.4, ay=0.9, bc_x=nat.TRANSMISSIVE, kind=""),
]


@pytest.mark.parametrize("case", CASES, ids=lambda c: f"eq{c['eqn']}-{c['nx']}x{c['ny']}-{c['kind']}")
@pytest.mark.parametrize("dtype", [nat.F64, nat.F32])
@pytest.mark.parametrize("scheme", ORDERS)
def test_residual_parity(case, dtype, scheme):
    case = dict(case)
    kind = case.pop("kind")
    c, o = make(dtype, scheme=scheme, **case)
    q = state(o, kind, 4)
    if dtype == nat.F32:
        q = q.astype(np.float32).astype(np.float64)
    R_or = oracle.residual(o, q)
    with nat.Context(c) as ctx:
        R = host(ctx.residual(dev(q, c)))
    assert rel(R, R_or) <= (TOL64 if dtype == nat.F64 else TOL32)


@pytest.mark.parametrize("dtype", [nat.F64, nat.F32])
@pytest.mark.parametrize("nsteps", [1, 2, 7])
@pytest.mark.parametrize("scheme", ORDERS)
def test_fixed_steps(dtype, nsteps, scheme):
    c, o = make(dtype, scheme=scheme, eqn=nat.EULER, nx=40, ny=24, x1=10.0, y1=6.0)
    q0 = state(o, "vortex", 8)
    if dtype == nat.F32:
        q0 = q0.astype(np.float32).astype(np.float64)
    q_or, _, _ = oracle.run(o, q0, nsteps, 0.01)
    with nat.Context(c) as ctx:
        qd = dev(q0, c)
        ctx.step(qd, nsteps, 0.01)
        assert ctx.get_time()[1] == nsteps
        q = host(qd)
    assert rel(q, q_or) <= (TOL64 if dtype == nat.F64 else 1e-6)


@pytest.mark.parametrize("scheme", ORDERS)
def test_cfl_steps_land_on_t_end(scheme):
    c, o = make(nat.F64, scheme=scheme, eqn=nat.EULER, nx=48, ny=40, bc_x=nat.TRANSMISSIVE,
                bc_y=nat.TRANSMISSIVE, cfl=0.4)
    q0 = state(o, "4q", 2)
    t_end = 0.05
    q_or, n_or, t_or = oracle.run(o, q0, 100000, 0.0, t_end)
    with nat.Context(c) as ctx:
        qd = dev(q0, c)
        ctx.step(qd, n_or + 5, 0.0, t_end)
        t, n = ctx.get_time()
        q = host(qd)
    assert t == t_end == t_or and n == n_or
    assert rel(q, q_or) <= TOL64


@pytest.mark.parametrize("scheme", ORDERS)
def test_averages_are_conserved_on_periodic_grid(scheme):
    c, o = make(nat.F64, scheme=scheme, eqn=nat.EULER, nx=64, ny=48, x1=10.0, y1=7.5, cfl=0.4)
    q0 = state(o, "vortex", 5)
    with nat.Context(c) as ctx:
        qd = dev(q0, c)
        s0 = np.array(ctx.norms(qd)["sum_avg"])
        ctx.step(qd, 60)
        s1 = np.array(ctx.norms(qd)["sum_avg"])
    assert np.allclose(s1, s0, rtol=1e-13, atol=1e-12)


@pytest.mark.parametrize("scheme", ORDERS)
def test_four_quadrant_full_size_one_step(scheme):
    """The FV run of the equal-DOF comparison: 1536 x 1536 elements (the
    2,359,296 DOF of the 512^2 p = 2 CPR run), transmissive, CFL 0.4: one
    SSP-RK3 step at the CFL step size in FP64, against the oracle."""
    c, o = make(nat.F64, scheme=scheme, eqn=nat.EULER, nx=1536, ny=1536, bc_x=nat.TRANSMISSIVE,
                bc_y=nat.TRANSMISSIVE, cfl=0.4)
    x, y = oracle.point_coords(o)
    q0 = inputs.four_quadrant(x, y)
    q_or, n, _ = oracle.run(o, q0, 1)
    with nat.Context(c) as ctx:
        qd = dev(q0, c)
        ctx.step(qd, 1)
        q = host(qd)
    assert n == 1 and rel(q, q_or) <= TOL64


def test_fv_has_no_troubled_cell_limiter_or_adjoint():
    c, _ = make(nat.F64, eqn=nat.EULER, nx=8, ny=8)
    with nat.Context(c) as ctx:
        q = torch.ones(c.shape, dtype=torch.float64, device="cuda")
        with pytest.raises(nat.CprError):
            ctx.limit(q)
        with pytest.raises(nat.CprError):
            ctx.residual_vjp(q, q)
