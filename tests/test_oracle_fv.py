"""Pins of the oracle's FV scheme (Sec. 2.1 semi-discretisation, second-order
MUSCL reconstruction with minmod slopes of Sec. 2.6, Rusanov / upwind face
fluxes): each check follows from the mathematics of the scheme, not from the
oracle's own formulas."""
import numpy as np
import pytest

import oracle
from paper_1709_01619_gb300 import inputs


def fv(**kw):
    kw.setdefault("p", 0)
    kw.setdefault("scheme", oracle.FV_MUSCL)
    return oracle.Config(**kw)


@pytest.mark.parametrize("bc", [oracle.PERIODIC, oracle.TRANSMISSIVE])
def test_freestream_is_steady(bc):
    for eqn in (oracle.EULER, oracle.ADVECTION):
        c = fv(eqn=eqn, nx=13, ny=9, bc_x=bc, bc_y=bc, x1=2.0, y1=1.5)
        x, y = oracle.point_coords(c)
        q = inputs.freestream(x) if eqn == oracle.EULER else np.full((1,) + x.shape, 0.7)
        assert np.abs(oracle.residual(c, q)).max() <= 1e-13


def test_averages_sum_is_conserved_on_periodic_grid():
    c = fv(eqn=oracle.EULER, nx=24, ny=20, x1=10.0, y1=10.0, cfl=0.4)
    x, y = oracle.point_coords(c)
    q = inputs.perturbed(inputs.vortex(x, y, eps=5.0), 3, 0.05)
    s0 = q.reshape(4, -1).sum(axis=1)
    q1, _, _ = oracle.run(c, q, 20)
    s1 = q1.reshape(4, -1).sum(axis=1)
    assert np.allclose(s1, s0, rtol=1e-13, atol=1e-12)


@pytest.mark.parametrize("flux", [oracle.UPWIND, oracle.RUSANOV])
def test_linear_data_is_reconstructed_exactly(flux):
    """On q = a + b x + c y the limited slopes are the exact slopes away from
    the boundary, both face states equal the face value, and R = -(ax b + ay c)
    in every element at least two away from a transmissive boundary."""
    c = fv(eqn=oracle.ADVECTION, nx=12, ny=11, flux=flux, ax=0.7, ay=-1.3, x1=3.0, y1=2.0,
           bc_x=oracle.TRANSMISSIVE, bc_y=oracle.TRANSMISSIVE)
    x, y = oracle.point_coords(c)
    b, cc = 0.9, -0.4
    q = (1.5 + b * x + cc * y)[None]
    R = oracle.residual(c, q).reshape(c.ny, c.nx)
    inner = R[2:-2, 2:-2]
    assert np.allclose(inner, -(0.7 * b - 1.3 * cc), rtol=0, atol=1e-12)


def test_zigzag_reduces_to_first_order_upwind():
    """Alternating data has a local extremum in every element: minmod sets
    every slope to zero and the scheme is first-order upwind,
    R_i = -a (q_i - q_{i-1}) / h for a > 0."""
    nx, ny, a, L = 16, 3, 1.7, 4.0
    c = fv(eqn=oracle.ADVECTION, nx=nx, ny=ny, flux=oracle.UPWIND, ax=a, ay=0.0, x1=L, y1=1.0)
    ii = np.tile(np.arange(nx), ny)
    q = (2.0 + (-1.0) ** ii + 0.1 * (ii % 3))[None].astype(float)
    R = oracle.residual(c, q).reshape(ny, nx)
    qq = q.reshape(ny, nx)
    expect = -a * (qq - np.roll(qq, 1, axis=1)) / (L / nx)
    assert np.allclose(R, expect, rtol=0, atol=1e-12)


@pytest.mark.parametrize("a", [1.3, -0.8])
def test_convex_increasing_data_gives_the_textbook_stencils(a):
    """For increasing data with increasing differences, minmod picks the
    backward difference: with a > 0 the upwind face state q_i + (q_i -
    q_{i-1})/2 gives R_i = -a (3 q_i - 4 q_{i-1} + q_{i-2}) / (2h); with a < 0
    the state q_{i+1} - (q_{i+1} - q_i)/2 gives the central difference
    R_i = -a (q_{i+1} - q_{i-1}) / (2h)."""
    nx, ny, L = 20, 2, 2.0
    h = L / nx
    c = fv(eqn=oracle.ADVECTION, nx=nx, ny=ny, flux=oracle.UPWIND, ax=a, ay=0.0, x1=L, y1=1.0,
           bc_x=oracle.TRANSMISSIVE)
    i = np.arange(nx, dtype=float)
    row = 0.5 + 0.3 * i + 0.05 * i * i + 0.004 * i ** 3
    q = np.tile(row, ny)[None]
    R = oracle.residual(c, q).reshape(ny, nx)[0]
    k = np.arange(2, nx - 2)
    if a > 0:
        expect = -a * (3 * row[k] - 4 * row[k - 1] + row[k - 2]) / (2 * h)
    else:
        expect = -a * (row[k + 1] - row[k - 1]) / (2 * h)
    assert np.allclose(R[k], expect, rtol=0, atol=1e-12)


def test_one_dimensional_step_stays_total_variation_diminishing():
    """MUSCL with minmod and SSP-RK3 at CFL 0.4 is TVD for linear advection:
    the total variation never grows and no new extrema appear."""
    nx, ny = 64, 2
    c = fv(eqn=oracle.ADVECTION, nx=nx, ny=ny, flux=oracle.UPWIND, ax=1.0, ay=0.0, x1=1.0, y1=0.1,
           cfl=0.4)
    x, y = oracle.point_coords(c)
    q = np.where((x > 0.2) & (x < 0.5), 2.0, 1.0)[None]
    dt = 0.4 * (1.0 / nx)
    tv0 = np.abs(np.diff(q.reshape(ny, nx), axis=1, append=q.reshape(ny, nx)[:, :1])).sum()
    for _ in range(40):
        q = oracle.rk3_step(c, q, dt)
        qq = q.reshape(ny, nx)
        tv = np.abs(np.diff(qq, axis=1, append=qq[:, :1])).sum()
        assert tv <= tv0 + 1e-12
        assert qq.min() >= 1.0 - 1e-12 and qq.max() <= 2.0 + 1e-12
        tv0 = tv


def test_convergence_on_smooth_advection():
    """sin 2 pi x sin 2 pi y advected to t = 0.125: minmod clips the slopes at
    the smooth extrema (lines here), so the scheme is second order away from
    them and the global orders settle near 1.5 (L2) and above it in L1; a
    first-order method gives 1."""
    errs1, errs2 = [], []
    for n in (32, 64):
        c = fv(eqn=oracle.ADVECTION, nx=n, ny=n, flux=oracle.UPWIND, ax=1.0, ay=1.0)
        q0 = oracle.exact_averages(c, "advection", 0.0).reshape(1, -1, 1)
        nsteps = n // 4                       # dt = 0.5 h
        q, _, _ = oracle.run(c, q0, nsteps, 0.125 / nsteps)
        d = q.reshape(-1) - oracle.exact_averages(c, "advection", 0.125).reshape(-1)
        errs1.append(np.abs(d).mean())
        errs2.append(np.sqrt(np.mean(d * d)))
    assert np.log2(errs2[0] / errs2[1]) >= 1.4, errs2
    assert np.log2(errs1[0] / errs1[1]) >= 1.45, errs1


def test_four_quadrant_keeps_diagonal_symmetry():
    n = 24
    c = fv(eqn=oracle.EULER, nx=n, ny=n, bc_x=oracle.TRANSMISSIVE, bc_y=oracle.TRANSMISSIVE, cfl=0.4)
    x, y = oracle.point_coords(c)
    q = inputs.four_quadrant(x, y)
    q, _, _ = oracle.run(c, q, 10)
    g = q.reshape(4, n, n)                     # [v, j, i]
    gt = g.transpose(0, 2, 1)
    assert np.allclose(g[0], gt[0], atol=1e-12)
    assert np.allclose(g[1], gt[2], atol=1e-12)
    assert np.allclose(g[2], gt[1], atol=1e-12)
    assert np.allclose(g[3], gt[3], atol=1e-12)
    assert (g[0] > 0).all()


def test_fv_rejects_limiter_and_nonzero_order():
    x = np.zeros(4 * 16)
    with pytest.raises(ValueError):
        oracle.residual(fv(eqn=oracle.EULER, nx=4, ny=4, limiter=1), x)
    with pytest.raises(ValueError):
        oracle.residual(fv(eqn=oracle.EULER, nx=4, ny=4, p=1), np.zeros(4 * 16 * 4))
