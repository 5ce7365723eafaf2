"""Pins of the oracle's third-order MUSCL finite-volume scheme (Sec. 2.1
semi-discretisation, third-order MUSCL reconstruction of Sec. 2.6 read as
van Leer's kappa = 1/3 scheme with minmod compression b = 4).

The checks follow from what a third-order limited reconstruction must do,
not from the oracle's own formula: freestream and conservation, exactness
for the averages of a parabola (the defining property of the
kappa = 1/3 reconstruction), reduction to first-order upwind on zigzag
data, face states bounded by the neighbouring averages (recovered from the
residual), total variation diminishing steps and the diagonal symmetry of
the four-quadrant problem."""
import numpy as np
import pytest

import oracle
from paper_1709_01619_gb300 import inputs


def fv3(**kw):
    kw.setdefault("p", 0)
    kw.setdefault("scheme", oracle.FV_MUSCL3)
    return oracle.Config(**kw)


@pytest.mark.parametrize("bc", [oracle.PERIODIC, oracle.TRANSMISSIVE])
def test_freestream_is_steady(bc):
    for eqn in (oracle.EULER, oracle.ADVECTION):
        c = fv3(eqn=eqn, nx=13, ny=9, bc_x=bc, bc_y=bc, x1=2.0, y1=1.5)
        x, y = oracle.point_coords(c)
        q = inputs.freestream(x) if eqn == oracle.EULER else np.full((1,) + x.shape, 0.7)
        assert np.abs(oracle.residual(c, q)).max() <= 1e-13


def test_averages_sum_is_conserved_on_periodic_grid():
    c = fv3(eqn=oracle.EULER, nx=24, ny=20, x1=10.0, y1=10.0, cfl=0.4)
    x, y = oracle.point_coords(c)
    q = inputs.perturbed(inputs.vortex(x, y, eps=5.0), 3, 0.05)
    s0 = q.reshape(4, -1).sum(axis=1)
    q1, _, _ = oracle.run(c, q, 20)
    assert np.allclose(q1.reshape(4, -1).sum(axis=1), s0, rtol=1e-13, atol=1e-12)


def upwind_face_states(c, q, a, h):
    """The upwind face states q^-_{i+1/2}, i = 0..nx-1, of a one-row advection
    problem with a > 0, recovered from the residual
    R_i = -a (q^-_{i+1/2} - q^-_{i-1/2}) / h by a running sum from the
    transmissive left boundary, where the ghost elements repeat q_0 and so
    q^-_{-1/2} = q_0."""
    R = oracle.residual(c, q).reshape(-1)
    return q.reshape(-1)[0] - np.cumsum(h * R / a)


def downwind_face_states(c, q, a, h):
    """The same for a < 0: the upwind states are q^+_{i-1/2}, recovered from
    the transmissive right boundary (q^+_{nx-1/2} = q_{nx-1}); entry i is
    q^+_{i-1/2}."""
    R = oracle.residual(c, q).reshape(-1)
    return q.reshape(-1)[-1] + np.cumsum((h * R / a)[::-1])[::-1]


def test_parabola_averages_give_exact_face_values():
    """Averages of the increasing parabola q = al + be x + ga x^2 over cells
    of width h: a third-order reconstruction returns the parabola's point
    value at every face where the limiter is inactive (the one-sided
    differences are within a factor 4 of each other here); the second-order
    one is off by 2/3 ga h^2."""
    nx, L, a = 24, 2.0, 1.1
    h = L / nx
    al, be, ga = 0.3, 0.8, 0.35
    xc = (np.arange(nx) + 0.5) * h
    avg = (al + be * xc + ga * (xc ** 2 + h * h / 12.0))[None]
    kw = dict(eqn=oracle.ADVECTION, nx=nx, ny=1, flux=oracle.UPWIND, ax=a, ay=0.0, x1=L, y1=1.0,
              bc_x=oracle.TRANSMISSIVE)
    xf = xc + 0.5 * h
    exact = al + be * xf + ga * xf ** 2
    k = np.arange(2, nx - 2)
    face3 = upwind_face_states(fv3(**kw), avg, a, h)
    assert np.allclose(face3[k], exact[k], rtol=0, atol=1e-12)
    face2 = upwind_face_states(oracle.Config(p=0, scheme=oracle.FV_MUSCL, **kw), avg, a, h)
    assert np.allclose(face2[k] - exact[k], -2.0 / 3.0 * ga * h * h, rtol=0, atol=1e-12)
    # the other side of each face, through the residual of a < 0
    kw["ax"] = -a
    xl = xc - 0.5 * h
    exact_l = al + be * xl + ga * xl ** 2
    down = downwind_face_states(fv3(**kw), avg, -a, h)
    assert np.allclose(down[k], exact_l[k], rtol=0, atol=1e-12)


@pytest.mark.parametrize("a", [1.0, -1.0])
def test_steep_side_reaches_the_neighbouring_average(a):
    """Compression b = (3 - kappa)/(1 - kappa) = 4: where the difference on
    the far side of an element is at least four times the one across the
    face, the face state equals the neighbouring average (the bound is
    attained), and for smaller ratios it stays strictly inside."""
    h, nx = 0.1, 12
    d = np.array([1.0, 1.0, 4.0, 1.0, 6.0, 1.0, 2.0, 1.0, 1.0, 1.0, 1.0])
    if a < 0:
        d = d[::-1]
    row = np.concatenate([[0.0], np.cumsum(d)])
    kw = dict(eqn=oracle.ADVECTION, nx=nx, ny=1, flux=oracle.UPWIND, ax=a, ay=0.0, x1=nx * h, y1=1.0,
              bc_x=oracle.TRANSMISSIVE)
    if a > 0:
        face = upwind_face_states(fv3(**kw), row[None].copy(), a, h)   # q^-_{i+1/2}
        dm, dp = np.diff(row)[:-1], np.diff(row)[1:]                 # element i = 1..nx-2
        own, nb, f = row[1:-1], row[2:], face[1:-1]
    else:
        face = downwind_face_states(fv3(**kw), row[None].copy(), a, h)  # q^+_{i-1/2}
        dm, dp = np.diff(row)[:-1], np.diff(row)[1:]
        own, nb, f = row[1:-1], row[:-2], face[1:-1]
        dm, dp = dp, dm
    at = dm >= 4 * dp
    assert at.sum() >= 2
    assert np.allclose(f[at], nb[at], rtol=0, atol=1e-12)
    inside = ~at
    assert (np.abs(f[inside] - nb[inside]) > 1e-3).all()


def test_zigzag_reduces_to_first_order_upwind():
    nx, ny, a, L = 16, 3, 1.7, 4.0
    c = fv3(eqn=oracle.ADVECTION, nx=nx, ny=ny, flux=oracle.UPWIND, ax=a, ay=0.0, x1=L, y1=1.0)
    ii = np.tile(np.arange(nx), ny)
    q = (2.0 + (-1.0) ** ii + 0.1 * (ii % 3))[None].astype(float)
    R = oracle.residual(c, q).reshape(ny, nx)
    qq = q.reshape(ny, nx)
    expect = -a * (qq - np.roll(qq, 1, axis=1)) / (L / nx)
    assert np.allclose(R, expect, rtol=0, atol=1e-12)


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_face_states_stay_between_neighbouring_averages(seed):
    """Random monotone data (one-sided differences varying by orders of
    magnitude): a bounded (TVD) reconstruction keeps every upwind face state
    q^-_{i+1/2} between q_i and q_{i+1}; the compression b = 4 is the largest
    that does."""
    rng = np.random.default_rng(seed)
    nx, ny, a, L = 40, 1, 1.0, 1.0
    h = L / nx
    steps = rng.uniform(0.0, 1.0, nx) ** 3                    # widely varying, some tiny
    row = np.cumsum(steps)
    c = fv3(eqn=oracle.ADVECTION, nx=nx, ny=ny, flux=oracle.UPWIND, ax=a, ay=0.0, x1=L, y1=1.0,
            bc_x=oracle.TRANSMISSIVE)
    face = upwind_face_states(c, row[None].copy(), a, h)
    lo = np.minimum(row[:-1], row[1:])
    hi = np.maximum(row[:-1], row[1:])
    assert (face[:-1] >= lo - 1e-12).all() and (face[:-1] <= hi + 1e-12).all()


def test_one_dimensional_step_stays_total_variation_diminishing():
    nx, ny = 64, 2
    c = fv3(eqn=oracle.ADVECTION, nx=nx, ny=ny, flux=oracle.UPWIND, ax=1.0, ay=0.0, x1=1.0, y1=0.1)
    x, y = oracle.point_coords(c)
    q = np.where((x > 0.2) & (x < 0.5), 2.0, 1.0)[None]
    dt = 0.3 * (1.0 / nx)
    qq = q.reshape(ny, nx)
    tv0 = np.abs(np.diff(qq, axis=1, append=qq[:, :1])).sum()
    for _ in range(40):
        q = oracle.rk3_step(c, q, dt)
        qq = q.reshape(ny, nx)
        tv = np.abs(np.diff(qq, axis=1, append=qq[:, :1])).sum()
        assert tv <= tv0 + 1e-12
        assert qq.min() >= 1.0 - 1e-12 and qq.max() <= 2.0 + 1e-12
        tv0 = tv


def test_four_quadrant_keeps_diagonal_symmetry():
    n = 24
    c = fv3(eqn=oracle.EULER, nx=n, ny=n, bc_x=oracle.TRANSMISSIVE, bc_y=oracle.TRANSMISSIVE, cfl=0.4)
    x, y = oracle.point_coords(c)
    q, _, _ = oracle.run(c, inputs.four_quadrant(x, y), 10)
    g = q.reshape(4, n, n)
    gt = g.transpose(0, 2, 1)
    assert np.allclose(g[0], gt[0], atol=1e-12)
    assert np.allclose(g[1], gt[2], atol=1e-12)
    assert np.allclose(g[2], gt[1], atol=1e-12)
    assert np.allclose(g[3], gt[3], atol=1e-12)
    assert (g[0] > 0).all()
