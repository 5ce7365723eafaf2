"""Discrete adjoint on the GPU: residual and RK3-step transposes against the
FP64 oracle, a dot-product check against central differences of the GPU
residual, and gradients through checkpointed rollouts (torch.autograd)."""
import numpy as np
import pytest
import torch

import oracle
from paper_1709_01619_gb300 import _native as nat
from paper_1709_01619_gb300 import adjoint, inputs

pytestmark = pytest.mark.gpu


def make(dtype=nat.F64, **kw):
    c = nat.Config(dtype=dtype, **kw)
    o = oracle.Config(eqn=c.eqn, nx=c.nx, ny=c.ny, p=c.p, x0=c.x0, x1=c.x1, y0=c.y0, y1=c.y1,
                      pts=c.pts, div=c.div, flux=c.flux, ax=c.ax, ay=c.ay, gamma=c.gamma,
                      bc_x=c.bc_x, bc_y=c.bc_y)
    return c, o


def rough(o, seed, noise=0.02):
    x, y = oracle.point_coords(o)
    q = inputs.vortex(x, y, eps=3.0, xc=0.5 * o.x1, yc=0.5 * o.y1, lx=o.x1, ly=o.y1)
    if o.eqn == oracle.ADVECTION:
        q = q[:1]
    return inputs.perturbed(q, seed, noise)


def dev(a, c):
    return torch.tensor(np.asarray(a).reshape(c.shape), dtype=c.torch_dtype, device="cuda")


def rel(a, b):
    a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
    return np.linalg.norm(a - b) / np.linalg.norm(b)


CASES = [(eqn, p, bc, flux) for eqn in (0, 1) for p in (1, 2, 3, 4) for bc in (0, 1)
         for flux in ((nat.RUSANOV,) if eqn == 1 else (nat.UPWIND, nat.RUSANOV))]


@pytest.mark.parametrize("case", CASES, ids=lambda c: f"eq{c[0]}-p{c[1]}-bc{c[2]}-f{c[3]}")
@pytest.mark.parametrize("dtype", [nat.F64, nat.F32])
def test_residual_vjp_matches_oracle(case, dtype):
    eqn, p, bc, flux = case
    c, o = make(dtype, eqn=eqn, nx=11, ny=9, p=p, x1=5.5, y1=4.5, bc_x=bc, bc_y=1 - bc, flux=flux,
                ax=0.8, ay=-0.5)
    q = rough(o, 1)
    w = np.random.default_rng(2).standard_normal(q.shape)
    if dtype == nat.F32:
        q = q.astype(np.float32).astype(np.float64)
        w = w.astype(np.float32).astype(np.float64)
    ref = oracle.residual_vjp(o, q, w)
    with nat.Context(c) as ctx:
        got = ctx.residual_vjp(dev(q, c), dev(w, c)).double().cpu().numpy()
    assert rel(got, ref) <= (1e-12 if dtype == nat.F64 else 1e-5)


@pytest.mark.parametrize("eqn", [0, 1])
def test_step_vjp_matches_oracle(eqn):
    c, o = make(nat.F64, eqn=eqn, nx=13, ny=10, p=3, x1=6.5, y1=5.0, ax=0.8, ay=-0.5)
    q = rough(o, 3)
    w = np.random.default_rng(4).standard_normal(q.shape)
    ref = oracle.rk3_vjp(o, q, 0.01, w)
    with nat.Context(c) as ctx:
        got = ctx.step_vjp(dev(q, c), dev(w, c), 0.01).cpu().numpy()
        # cotangent arrays may alias
        wa = dev(w, c)
        ctx.step_vjp(dev(q, c), wa, 0.01, wa)
        assert rel(wa.cpu().numpy(), ref) <= 1e-12
    assert rel(got, ref) <= 1e-12


@pytest.mark.parametrize("eqn", [0, 1])
@pytest.mark.parametrize("dtype", [nat.F64, nat.F32])
def test_step_stages_and_their_vjp(eqn, dtype):
    """cpr_step_stages: the stage states and the new state of the Shu-Osher
    step (Sec. 4) against the oracle's residual composed in that order (FP64
    <= 1e-12, FP32 <= 1e-5); cpr_step_vjp_stages around them: cpr_step_vjp's
    result bit for bit (the same transposed residuals around the same stage
    states) and, in FP64, the oracle's step adjoint to 1e-12; the argument
    rules."""
    c, o = make(dtype, eqn=eqn, nx=13, ny=10, p=3, x1=6.5, y1=5.0, ax=0.8, ay=-0.5)
    q = rough(o, 5)
    w = np.random.default_rng(6).standard_normal(q.shape)
    if dtype == nat.F32:
        q = q.astype(np.float32).astype(np.float64)
        w = w.astype(np.float32).astype(np.float64)
    dt = 0.01
    q1r = q + dt * oracle.residual(o, q)
    q2r = 0.75 * q + 0.25 * (q1r + dt * oracle.residual(o, q1r))
    qnr = q / 3.0 + (2.0 / 3.0) * (q2r + dt * oracle.residual(o, q2r))
    tol = 1e-12 if dtype == nat.F64 else 1e-5
    with nat.Context(c) as ctx:
        qd = dev(q, c)
        q1, q2, qn = (torch.empty_like(qd) for _ in range(3))
        ctx.step_stages(qd, q1, q2, qn, dt)
        for got, ref in ((q1, q1r), (q2, q2r), (qn, qnr)):
            assert rel(got.double().cpu().numpy(), ref) <= tol
        a = ctx.step_vjp_stages(qd, q1, q2, dev(w, c), dt)
        b = ctx.step_vjp(qd, dev(w, c), dt)
        assert torch.equal(a, b)
        if dtype == nat.F64:
            assert rel(a.cpu().numpy(), oracle.rk3_vjp(o, q, dt, w)) <= 1e-12
        wd = dev(w, c)
        for bad in ((qd, qd, q2, qn, dt), (qd, q1, q1, qn, dt), (qd, q1, q2, q2, dt), (qd, q1, q2, qn, 0.0)):
            with pytest.raises(nat.CprError):
                ctx.step_stages(*bad)
        for bad in ((qd, q1, q2, qd, dt), (qd, q1, wd, wd, dt), (qd, q1, q2, wd, float("nan"))):
            with pytest.raises(nat.CprError):
                ctx.step_vjp_stages(*bad, qbar_in=torch.empty_like(qd))


def test_vjp_dot_product_with_gpu_residual_differences():
    c, o = make(nat.F64, eqn=1, nx=10, ny=12, p=2, x1=5.0, y1=6.0, bc_x=1)
    q = dev(rough(o, 5), c)
    rng = np.random.default_rng(6)
    with nat.Context(c) as ctx:
        for _ in range(3):
            v = dev(rng.standard_normal(c.shape), c)
            w = dev(rng.standard_normal(c.shape), c)
            h = 1e-6
            jv = (ctx.residual(q + h * v) - ctx.residual(q - h * v)) / (2 * h)
            lhs = float((jv * w).sum())
            rhs = float((v * ctx.residual_vjp(q, w)).sum())
            assert abs(lhs - rhs) <= 1e-7 * abs(rhs)


def test_rollout_gradient_matches_central_differences():
    c, _ = make(nat.F64, eqn=1, nx=12, ny=10, p=3, x1=10.0, y1=8.0, cfl=0.08)
    with nat.Context(c) as ctx:
        x, y = ctx.point_coords()
        q0 = torch.tensor(inputs.vortex(x, y, eps=4.0, xc=5.0, yc=4.0, ly=8.0), device="cuda")
        qt = torch.tensor(inputs.vortex(x, y, eps=3.5, xc=5.0, yc=4.0, ly=8.0), device="cuda")
        W = adjoint.quadrature_weights(ctx)
        nsteps, dt = 10, 0.01

        def J(q):
            qN = adjoint.rollout(q, ctx, nsteps, dt, every=4)
            return 0.5 * (W * (qN - qt) ** 2).sum()

        q0r = q0.clone().requires_grad_(True)
        J(q0r).backward()
        g = q0r.grad
        rng = np.random.default_rng(7)
        for _ in range(4):
            d = torch.tensor(rng.standard_normal(c.shape), device="cuda")
            h = 1e-5
            with torch.no_grad():
                fd = (J(q0 + h * d) - J(q0 - h * d)) / (2 * h)
            assert float((g * d).sum()) == pytest.approx(float(fd), rel=1e-6)


def test_fp32_gradient_against_oracle_adjoint_16x16():
    """FP32 gradient of the misfit through 8 steps vs the FP64 oracle's
    discrete adjoint chain on 16 x 16, p = 3."""
    c, o = make(nat.F32, eqn=1, nx=16, ny=16, p=3, x1=10.0, y1=10.0)
    x, y = oracle.point_coords(o)
    q0 = inputs.vortex(x, y, eps=5.0).astype(np.float32).astype(np.float64)
    qt = inputs.vortex(x, y, eps=4.5)
    nsteps, dt = 8, 0.01
    states = [q0]
    for _ in range(nsteps):
        states.append(oracle.rk3_step(o, states[-1], dt))
    t = oracle.tables(3, oracle.GAUSS)
    hx = hy = 10.0 / 16
    Wp = (hx * hy / 4) * np.outer(t["w"], t["w"]).reshape(16)
    gbar = Wp[None, None, :] * (states[-1] - qt)
    for s in reversed(range(nsteps)):
        gbar = oracle.rk3_vjp(o, states[s], dt, gbar)
    with nat.Context(c) as ctx:
        q0d = dev(q0, c).requires_grad_(True)
        qN = adjoint.rollout(q0d, ctx, nsteps, dt, every=3)
        W = adjoint.quadrature_weights(ctx)
        (0.5 * (W * (qN - dev(qt, c)) ** 2).sum()).backward()
        g = q0d.grad.double().cpu().numpy()
    assert rel(g, gbar) <= 1e-4


def test_config5_gradient_full_size_vs_fp64_differences():
    """Adjoint workload at full size: J = 1/2 sum W (q_N - q_t)^2 for the
    Euler vortex (strength 5) on [0,10]^2, 256 x 256, p = 3, 400 SSP-RK3 steps
    of dt = 7e-4 (t = 0.28, CFL 0.07 at the vortex's largest signal speed of
    about 3.9; 400 stable steps cannot reach t = 2),
    checkpoints every 20 steps; q_t is the forward solution from the vortex
    of strength 4.5.

    (1) The FP64 adjoint gradient g projected on 32 random Gaussian
    directions d against central differences of J (h = 1e-4) from the FP64
    solver.  For unit-variance Gaussian d the projection g.d has standard
    deviation |g|, its natural scale: the error |g.d - fd| stays below
    2e-5 |g| (the O(h^2) truncation), and below 1e-4 |g.d| wherever the
    projection is not close to zero (|g.d| > 0.2 |g|).
    (2) The FP32 adjoint gradient: its projections against the same FP64
    central differences (FP32 rounding accumulated over 1200 stages and
    their adjoints: within 3e-4 |g|), and against the FP64 gradient, relative
    L2 over the whole vector (5.4e-5 seen; bound 2e-4)."""
    n, nsteps, dt = 256, 400, 7e-4
    c32 = nat.Config(dtype=nat.F32, eqn=nat.EULER, nx=n, ny=n, p=3, x1=10.0, y1=10.0)
    c64 = nat.Config(dtype=nat.F64, eqn=nat.EULER, nx=n, ny=n, p=3, x1=10.0, y1=10.0)
    with nat.Context(c64) as ctx64, nat.Context(c32) as ctx32:
        x, y = ctx64.point_coords()
        q0 = torch.tensor(inputs.vortex(x, y, eps=5.0), device="cuda")
        qt = torch.tensor(inputs.vortex(x, y, eps=4.5), device="cuda")
        ctx64.step(qt, nsteps, dt)
        W64 = adjoint.quadrature_weights(ctx64)

        def J64(q):
            q = q.clone()
            ctx64.step(q, nsteps, dt)
            return float(0.5 * (W64 * (q - qt) ** 2).sum())

        q64 = q0.clone().requires_grad_(True)
        qN = adjoint.rollout(q64, ctx64, nsteps, dt, every=20)
        (0.5 * (W64 * (qN - qt) ** 2).sum()).backward()
        g64 = q64.grad.clone()

        q32 = q0.float().requires_grad_(True)
        qN = adjoint.rollout(q32, ctx32, nsteps, dt, every=20)
        W32 = adjoint.quadrature_weights(ctx32)
        (0.5 * (W32 * (qN - qt.float()) ** 2).sum()).backward()
        g32 = q32.grad.double()
        assert float((g32 - g64).norm() / g64.norm()) <= 2e-4

        rng = np.random.default_rng(5)
        h = 1e-4
        gn = float(g64.norm())
        big = 0
        for _ in range(32):
            d = torch.tensor(rng.standard_normal(c64.shape), device="cuda")
            fd = (J64(q0 + h * d) - J64(q0 - h * d)) / (2 * h)
            p64 = float((g64 * d).sum())
            assert abs(p64 - fd) <= 2e-5 * gn
            if abs(p64) > 0.2 * gn:
                big += 1
                assert abs(p64 - fd) <= 1e-4 * abs(p64)
            assert abs(float((g32 * d).sum()) - fd) <= 3e-4 * gn
        assert big >= 16  # most projections are not near zero
