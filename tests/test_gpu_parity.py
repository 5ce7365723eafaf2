"""CUDA path vs the FP64 oracle, element by element, through the C ABI.

Tolerances (relative L2 over every value, unless stated):
  FP64 kernels vs FP64 oracle  <= 1e-12  (rounding order and fused multiply-add
                                          only; the target the method states)
  FP32 kernels vs FP64 oracle  <= 1e-5   (the FP32 state tolerance; residual
                                          checks use rough inputs so that R is
                                          not a small difference of large terms)
Limiter marks are integers and compared exactly wherever the oracle's marking
margin is farther from zero than the arithmetic can move it.
Grids span several 8x8 element tiles with ragged tails (19 x 13 and similar).
"""
import math

import numpy as np
import pytest
import torch

import oracle
from paper_1709_01619_gb300 import _native as nat
from paper_1709_01619_gb300 import inputs

pytestmark = pytest.mark.gpu

TOL64 = 1e-12
TOL32 = 1e-5


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm((a - b).ravel()) / max(np.linalg.norm(b.ravel()), 1e-300))


def make(dtype=nat.F64, **kw):
    c = nat.Config(dtype=dtype, **kw)
    o = oracle.Config(eqn=c.eqn, nx=c.nx, ny=c.ny, p=c.p, x0=c.x0, x1=c.x1, y0=c.y0, y1=c.y1,
                      pts=c.pts, div=c.div, flux=c.flux, ax=c.ax, ay=c.ay, gamma=c.gamma,
                      bc_x=c.bc_x, bc_y=c.bc_y, limiter=c.limiter, tvb_M=c.tvb_M,
                      lim_eps=c.lim_eps, cfl=c.cfl)
    return c, o


def to_dev(q, c):
    return torch.tensor(np.asarray(q).reshape(c.shape), dtype=c.torch_dtype, device="cuda")


def host(t):
    return t.detach().double().cpu().numpy()


def rough_state(o, seed, noise=0.01):
    x, y = oracle.point_coords(o)
    if o.eqn == oracle.ADVECTION:
        return np.random.default_rng(seed).standard_normal((1, o.ne, o.n * o.n))
    q = inputs.vortex(x, y, eps=3.0, xc=0.5 * (o.x0 + o.x1), yc=0.5 * (o.y0 + o.y1),
                      lx=o.x1 - o.x0, ly=o.y1 - o.y0)
    return inputs.perturbed(q, seed, noise)


# ---------------------------------------------------------------------------
# coordinates and tables
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("pts", [0, 1])
@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_point_coords_match_oracle(p, pts):
    c, o = make(eqn=nat.EULER, nx=11, ny=7, p=p, pts=pts, x0=-1.0, x1=2.0, y0=0.5, y1=3.0)
    with nat.Context(c) as ctx:
        x, y = ctx.point_coords()
    xo, yo = oracle.point_coords(o)
    np.testing.assert_allclose(x, xo, rtol=0, atol=4e-16 * 3)
    np.testing.assert_allclose(y, yo, rtol=0, atol=4e-16 * 3)


# ---------------------------------------------------------------------------
# residual
# ---------------------------------------------------------------------------
RES_CASES = []
for p in (1, 2, 3, 4):
    for pts in (0, 1):
        for div in (0, 1):
            RES_CASES.append(dict(eqn=nat.EULER, p=p, pts=pts, div=div, bc=0))
        RES_CASES.append(dict(eqn=nat.EULER, p=p, pts=pts, div=0, bc=1))
        RES_CASES.append(dict(eqn=nat.ADVECTION, p=p, pts=pts, div=0, bc=0, flux=nat.UPWIND))
        RES_CASES.append(dict(eqn=nat.ADVECTION, p=p, pts=pts, div=1, bc=1, flux=nat.RUSANOV))


def _res_cfg(case, dtype, nx=19, ny=13):
    return make(dtype=dtype, eqn=case["eqn"], nx=nx, ny=ny, p=case["p"], pts=case["pts"],
                div=case["div"], flux=case.get("flux", nat.RUSANOV), bc_x=case["bc"], bc_y=case["bc"],
                x0=0.0, x1=9.5, y0=0.0, y1=6.5, ax=0.8, ay=-1.3)


@pytest.mark.parametrize("case", RES_CASES, ids=lambda c: "-".join(f"{k}{v}" for k, v in c.items()))
def test_residual_parity_fp64(case):
    c, o = _res_cfg(case, nat.F64)
    q = rough_state(o, 1)
    R_or = oracle.residual(o, q)
    with nat.Context(c) as ctx:
        R = host(ctx.residual(to_dev(q, c)))
    assert rel_l2(R, R_or) <= TOL64
    assert np.abs(R - R_or).max() <= 1e-11 * np.abs(R_or).max()


@pytest.mark.parametrize("case", RES_CASES[::3], ids=lambda c: "-".join(f"{k}{v}" for k, v in c.items()))
def test_residual_parity_fp32(case):
    c, o = _res_cfg(case, nat.F32)
    q = rough_state(o, 2, noise=0.05).astype(np.float32).astype(np.float64)
    R_or = oracle.residual(o, q)
    with nat.Context(c) as ctx:
        R = host(ctx.residual(to_dev(q, c)))
    assert rel_l2(R, R_or) <= TOL32


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_fp32_residual_on_both_sides_of_the_two_ctas_per_sm_grid(p):
    """The FP32 Euler / LP / Rusanov stage kernel has an instantiation for
    grids that fit the device at once (at most two 8x8-element CTAs per SM,
    four 8x4-element ones for p = 4; more registers) and one for larger
    grids: a grid just past that bound and a small one both match the
    oracle."""
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    ty = 2 * sms // 24 + 2
    assert 24 * ty > 2 * sms
    for nx, ny in ((19, 13), (8 * 24, 8 * ty - 3)):
        c, o = make(dtype=nat.F32, eqn=nat.EULER, nx=nx, ny=ny, p=p, x1=10.0, y1=10.0 * ny / nx)
        q = rough_state(o, 4, noise=0.05).astype(np.float32).astype(np.float64)
        R_or = oracle.residual(o, q)
        with nat.Context(c) as ctx:
            R = host(ctx.residual(to_dev(q, c)))
        assert rel_l2(R, R_or) <= TOL32, (nx, ny)


@pytest.mark.parametrize("shape", [(1, 1), (1, 5), (5, 1), (8, 8), (9, 17), (16, 3)])
def test_residual_degenerate_and_tile_edge_grids(shape):
    for bc in (0, 1):
        c, o = make(eqn=nat.EULER, nx=shape[0], ny=shape[1], p=2, bc_x=bc, bc_y=1 - bc,
                    x1=float(shape[0]), y1=float(shape[1]))
        q = rough_state(o, 3)
        with nat.Context(c) as ctx:
            R = host(ctx.residual(to_dev(q, c)))
        assert rel_l2(R, oracle.residual(o, q)) <= TOL64


def test_freestream_residual_is_roundoff():
    """A uniform state has R = 0; the computed R is rounding only, bounded by
    a few units of rounding of the largest term: (2/h) * max row sum |D| *
    max |f| (each point sums N products of that size)."""
    c0, o = make(eqn=nat.EULER, nx=21, ny=10, p=3, bc_x=1, x1=2.0, y1=1.0)
    x, _ = oracle.point_coords(o)
    q = inputs.freestream(x)
    D = oracle.tables(3, oracle.GAUSS)["D"]
    fmax = 2.5   # largest flux component of this state: (e + p) u = 3.44 * 0.7 = 2.41
    scale = (2.0 / min(2.0 / 21, 1.0 / 10)) * np.abs(D).sum(axis=1).max() * fmax
    for dtype, eps in ((nat.F64, 2.0 ** -53), (nat.F32, 2.0 ** -24)):
        c, _ = make(dtype=dtype, eqn=nat.EULER, nx=21, ny=10, p=3, bc_x=1, x1=2.0, y1=1.0)
        with nat.Context(c) as ctx:
            R = host(ctx.residual(to_dev(q, c)))
        assert np.abs(R).max() < 8 * eps * scale


# ---------------------------------------------------------------------------
# RK3 steps
# ---------------------------------------------------------------------------
def test_config1_full_run_fp64():
    """2D linear advection on [0,1]^2, 16x16, p=2 Gauss points, upwind, CFL 0.1
    to t=1 in equal steps, FP64: the whole run against the oracle."""
    c, o = make(eqn=nat.ADVECTION, nx=16, ny=16, p=2, flux=nat.UPWIND, ax=1.0, ay=1.0, cfl=0.1)
    x, y = oracle.point_coords(o)
    q0 = inputs.advection_sine(x, y)
    dt0 = 0.1 * (1.0 / 16) / math.sqrt(2.0)
    n = math.ceil(1.0 / dt0)
    assert n == 227
    q_or, _, _ = oracle.run(o, q0, n, 1.0 / n)
    with nat.Context(c) as ctx:
        qd = to_dev(q0, c)
        ctx.step(qd, n, 1.0 / n)
        q = host(qd)
        t, steps = ctx.get_time()
    assert steps == n and t == pytest.approx(1.0, abs=1e-13)
    assert rel_l2(q, q_or) <= TOL64
    ex = oracle.exact_averages(o, "advection", 1.0)
    e_gpu, e_or = oracle.rho_avg_error(o, q, ex), oracle.rho_avg_error(o, q_or, ex)
    assert e_gpu == pytest.approx(e_or, rel=1e-9)


def test_config1_full_run_fp32():
    """The same advection run in FP32 (compensated increment form): all 227
    steps against the FP64 oracle within the FP32 bound."""
    c, o = make(dtype=nat.F32, eqn=nat.ADVECTION, nx=16, ny=16, p=2, flux=nat.UPWIND, ax=1.0, ay=1.0,
                cfl=0.1)
    x, y = oracle.point_coords(o)
    q0 = inputs.advection_sine(x, y).astype(np.float32).astype(np.float64)
    n = 227
    q_or, _, _ = oracle.run(o, q0, n, 1.0 / n)
    with nat.Context(c) as ctx:
        qd = to_dev(q0, c)
        ctx.step(qd, n, 1.0 / n)
        q = host(qd)
        assert ctx.get_time()[1] == n
    assert rel_l2(q, q_or) <= TOL32


def test_fp32_euler_two_hundred_cfl_steps():
    """Euler vortex on a ragged 19 x 13 grid, p = 3, 200 CFL steps in FP32
    against the FP64 oracle (the step sizes are the device's own, from its
    FP64 reduction of the FP32 state, so the two runs also agree in time)."""
    c, o = make(dtype=nat.F32, eqn=nat.EULER, nx=19, ny=13, p=3, x1=10.0, y1=7.0, cfl=0.08)
    x, y = oracle.point_coords(o)
    q0 = inputs.vortex(x, y, eps=5.0, xc=5.0, yc=3.5, ly=7.0).astype(np.float32).astype(np.float64)
    q_or, n_or, t_or = oracle.run(o, q0, 200)
    with nat.Context(c) as ctx:
        qd = to_dev(q0, c)
        ctx.step(qd, 200)
        q = host(qd)
        t, steps = ctx.get_time()
    assert steps == n_or == 200
    assert t == pytest.approx(t_or, rel=1e-6)
    assert rel_l2(q, q_or) <= TOL32


@pytest.mark.parametrize("dtype", [nat.F64, nat.F32])
def test_config2_fixed_steps(dtype):
    """Euler isentropic vortex, 128x128, p=3, periodic [0,10]^2, CFL steps: the
    full-size state after a fixed step count, in the launch configuration the
    benchmark times (cpr_step with device-side CFL steps)."""
    c, o = make(dtype=dtype, eqn=nat.EULER, nx=128, ny=128, p=3, x1=10.0, y1=10.0, cfl=0.08)
    x, y = oracle.point_coords(o)
    q0 = inputs.vortex(x, y, eps=5.0)
    if dtype == nat.F32:
        q0 = q0.astype(np.float32).astype(np.float64)
    nsteps = 35  # one 32-step graph, then a two-step and a one-step graph
    q_or, n_or, t_or = oracle.run(o, q0, nsteps)
    with nat.Context(c) as ctx:
        qd = to_dev(q0, c)
        ctx.step(qd, nsteps)
        q = host(qd)
        t, steps = ctx.get_time()
    assert steps == n_or == nsteps
    assert t == pytest.approx(t_or, rel=1e-12 if dtype == nat.F64 else 1e-6)
    assert rel_l2(q, q_or) <= (TOL64 if dtype == nat.F64 else TOL32)


def test_cfl_steps_land_on_t_end():
    c, o = make(eqn=nat.EULER, nx=24, ny=20, p=2, x1=10.0, y1=10.0, cfl=0.1)
    x, y = oracle.point_coords(o)
    q0 = inputs.vortex(x, y, eps=5.0)
    t_end = 0.1234
    q_or, n_or, t_or = oracle.run(o, q0, 10000, 0.0, t_end)
    with nat.Context(c) as ctx:
        qd = to_dev(q0, c)
        ctx.step(qd, n_or + 7, 0.0, t_end)  # surplus steps must do nothing
        q = host(qd)
        t, steps = ctx.get_time()
    assert t_or == t_end and t == t_end
    assert steps == n_or
    assert rel_l2(q, q_or) <= TOL64


@pytest.mark.parametrize("nsteps", [1, 2, 3, 7, 8, 9, 17, 31, 32, 33, 66])
def test_fp32_increment_form_step_counts(nsteps):
    """FP32 runs without the limiter use the increment form of SSP-RK3 with a
    compensated state whose high part alternates between two buffers: every
    step count, odd or even, below, at and past the 32-step graph (the rest
    runs as two-step and one-step graphs), lands in the caller's array and
    matches the FP64 oracle."""
    c, o = make(dtype=nat.F32, eqn=nat.EULER, nx=19, ny=13, p=3, x1=10.0, y1=7.0, cfl=0.08)
    x, y = oracle.point_coords(o)
    q0 = inputs.vortex(x, y, eps=5.0, xc=5.0, yc=3.5, ly=7.0).astype(np.float32).astype(np.float64)
    q_or, _, _ = oracle.run(o, q0, nsteps, 0.01)
    with nat.Context(c) as ctx:
        qd = to_dev(q0, c)
        ctx.step(qd, nsteps, 0.01)
        q = host(qd)
        assert ctx.get_time()[1] == nsteps
    assert rel_l2(q, q_or) <= 1e-6


def test_fp32_cfl_run_to_t_end():
    c, o = make(dtype=nat.F32, eqn=nat.EULER, nx=24, ny=20, p=3, x1=10.0, y1=10.0, cfl=0.08)
    x, y = oracle.point_coords(o)
    q0 = inputs.vortex(x, y, eps=5.0).astype(np.float32).astype(np.float64)
    t_end = 0.25
    q_or, n_or, _ = oracle.run(o, q0, 10000, 0.0, t_end)
    with nat.Context(c) as ctx:
        qd = to_dev(q0, c)
        ctx.step(qd, n_or + 5, 0.0, t_end)
        q = host(qd)
        t, steps = ctx.get_time()
    assert t == t_end and steps == n_or
    assert rel_l2(q, q_or) <= 1e-6


def test_step_host_equals_step():
    c, o = make(eqn=nat.EULER, nx=19, ny=13, p=3, x1=10.0, y1=7.0, cfl=0.08)
    q0 = rough_state(o, 4, noise=0.0)
    with nat.Context(c) as ctx:
        qd = to_dev(q0, c)
        ctx.step(qd, 5, 0.01)
        a = host(qd)
    with nat.Context(c) as ctx:
        qh = torch.tensor(q0, dtype=torch.float64).contiguous().pin_memory()
        out = torch.empty_like(qh).pin_memory()
        ctx.step_host(qh, out, 5, 0.01)
        b = out.numpy()
    np.testing.assert_array_equal(a, b)


def test_zero_steps_is_a_noop():
    c, o = make(eqn=nat.EULER, nx=9, ny=9, p=2, x1=10.0, y1=10.0)
    q0 = rough_state(o, 5)
    with nat.Context(c) as ctx:
        qd = to_dev(q0, c)
        ctx.step(qd, 0)
        assert np.array_equal(host(qd), q0)
        assert ctx.get_time() == (0.0, 0)


# ---------------------------------------------------------------------------
# averages, norms, limiter
# ---------------------------------------------------------------------------
def test_averages_and_norms_parity():
    c, o = make(eqn=nat.EULER, nx=19, ny=13, p=3, x1=10.0, y1=7.0)
    q = rough_state(o, 6)
    ref = rough_state(o, 7)
    with nat.Context(c) as ctx:
        qd = to_dev(q, c)
        avg = host(ctx.averages(qd))
        nr = ctx.norms(qd, to_dev(ref, c))
    np.testing.assert_allclose(avg, oracle.averages(o, q), rtol=1e-14, atol=1e-14)
    no = oracle.norms(o, q, ref)
    np.testing.assert_allclose(nr["sum_avg"], no["sum_avg"], rtol=1e-13)
    assert nr["l2_rel"] == pytest.approx(no["l2_rel"], rel=1e-12)
    assert nr["max_wave"] == pytest.approx(no["max_wave"], rel=1e-14)
    assert nr["n_nonphys"] == 0


def test_nonphysical_points_are_counted():
    c, o = make(eqn=nat.EULER, nx=9, ny=9, p=2, x1=10.0, y1=10.0)
    q = rough_state(o, 8).copy()
    q[0, 5, 3] = -0.1            # negative density
    q[3, 7, 0] = 0.0             # zero energy -> negative pressure
    q[1, 9, 4] = np.nan
    with nat.Context(c) as ctx:
        nr = ctx.norms(to_dev(q, c))
    assert nr["status"] == nat.CPR_ENONPHYS and nr["n_nonphys"] == 3


def _four_quadrant(o):
    x, y = oracle.point_coords(o)
    return inputs.four_quadrant(x, y)


@pytest.mark.parametrize("dtype", [nat.F64, nat.F32])
@pytest.mark.parametrize("pts", [0, 1])
def test_limiter_parity(dtype, pts):
    c, o = make(dtype=dtype, eqn=nat.EULER, nx=37, ny=29, p=2, pts=pts, bc_x=nat.TRANSMISSIVE,
                bc_y=nat.TRANSMISSIVE, limiter=1, tvb_M=50.0, lim_eps=1e-3)
    q = inputs.perturbed(_four_quadrant(o), 9, 2e-3)
    if dtype == nat.F32:
        q = q.astype(np.float32).astype(np.float64)
    q_or, marks_or, margin, cnt = oracle.limit(o, q)
    with nat.Context(c) as ctx:
        qd = to_dev(q, c)
        ctx.limit(qd)
        marks = ctx.get_marks()
        ql = host(qd)
        n_marked = ctx.norms(qd)["n_marked"]
    sure = np.abs(margin) > (1e-10 if dtype == nat.F64 else 1e-4)
    assert np.array_equal(marks[sure], marks_or[sure])
    assert n_marked == marks.sum()
    agree = marks == marks_or
    assert agree.mean() > 0.99 and cnt > 10
    V, ne, P = ql.shape
    a = ql[:, agree, :]
    b = q_or[:, agree, :]
    assert rel_l2(a, b) <= (TOL64 if dtype == nat.F64 else TOL32)


@pytest.mark.parametrize("dtype", [nat.F64, nat.F32])
@pytest.mark.parametrize("p", [1, 3, 4])
@pytest.mark.parametrize("eqn", [nat.EULER, nat.ADVECTION])
def test_limiter_parity_other_orders(eqn, p, dtype):
    """The limiter kernel (one thread per element and variable) for the
    other orders and for one variable: 41 x 23 elements (a ragged last
    block), periodic in x, transmissive in y."""
    kw = dict(flux=nat.UPWIND, ax=0.9, ay=-0.6) if eqn == nat.ADVECTION else {}
    c, o = make(dtype=dtype, eqn=eqn, nx=41, ny=23, p=p, bc_x=nat.PERIODIC, bc_y=nat.TRANSMISSIVE,
                limiter=1, tvb_M=20.0, lim_eps=1e-3, **kw)
    if eqn == nat.EULER:
        q = inputs.perturbed(_four_quadrant(o), 3 + p, 2e-3)
    else:
        x, y = oracle.point_coords(o)
        q = (np.where(x + 0.5 * y > 0.6, 1.0, 0.2) + 0.05 * np.sin(7 * x))[None]
    if dtype == nat.F32:
        q = q.astype(np.float32).astype(np.float64)
    q_or, marks_or, margin, cnt = oracle.limit(o, q)
    with nat.Context(c) as ctx:
        qd = to_dev(q, c)
        ctx.limit(qd)
        marks = ctx.get_marks()
        ql = host(qd)
        n_marked = ctx.norms(qd)["n_marked"]
    sure = np.abs(margin) > (1e-10 if dtype == nat.F64 else 1e-4)
    assert np.array_equal(marks[sure], marks_or[sure])
    assert n_marked == marks.sum() and cnt > 10
    agree = marks == marks_or
    assert agree.mean() > 0.99
    assert rel_l2(ql[:, agree, :], q_or[:, agree, :]) <= (TOL64 if dtype == nat.F64 else TOL32)


def test_steps_with_limiter_fp64():
    c, o = make(eqn=nat.EULER, nx=40, ny=40, p=2, bc_x=nat.TRANSMISSIVE, bc_y=nat.TRANSMISSIVE,
                limiter=1, tvb_M=50.0, lim_eps=1e-3, cfl=0.1)
    q0, _, _, _ = oracle.limit(o, _four_quadrant(o))
    q_or, n_or, _ = oracle.run(o, q0, 6, 2e-4)
    with nat.Context(c) as ctx:
        qd = to_dev(q0, c)
        ctx.step(qd, 6, 2e-4)
        q = host(qd)
    assert rel_l2(q, q_or) <= TOL64


def test_config3_full_size_one_step_fp64():
    """Four-quadrant Riemann problem, 512x512, p=2, TVB limiter, transmissive:
    one full-size SSP-RK3 step (limiter after every stage) vs the oracle."""
    c, o = make(eqn=nat.EULER, nx=512, ny=512, p=2, bc_x=nat.TRANSMISSIVE, bc_y=nat.TRANSMISSIVE,
                limiter=1, tvb_M=50.0, lim_eps=1e-3, cfl=0.1)
    q0, _, _, _ = oracle.limit(o, _four_quadrant(o))
    dt = oracle.dt(o, q0)
    q_or, _, _ = oracle.run(o, q0, 1, dt)
    with nat.Context(c) as ctx:
        qd = to_dev(q0, c)
        ctx.step(qd, 1, dt)
        q = host(qd)
    assert rel_l2(q, q_or) <= TOL64
