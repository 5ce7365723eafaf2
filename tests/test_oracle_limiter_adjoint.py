"""Pins of the oracle's troubled-cell limiter and its discrete adjoint.

Limiter (Sec. 2.6, Eq. 35, Algorithms 10-11): linear fields are fixed points,
marks exactly on the elements that contain a jump, limited values bounded by
the neighbouring averages and monotone across a step, averages preserved,
TVB bound and threshold behaviour.

Adjoint: the linearised residual against central differences of the
residual, and the transpose against the linearisation (dot-product test).
"""
import numpy as np
import pytest

from paper_1709_01619_gb300 import inputs


def _cfg(orc, **kw):
    base = dict(eqn=orc.EULER, nx=8, ny=6, p=2, limiter=1, tvb_M=0.0, lim_eps=1e-3)
    base.update(kw)
    return orc.Config(**base)


@pytest.mark.parametrize("pts", [0, 1])
@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_linear_fields_are_fixed_points(orc, p, pts):
    """Edge points see the tangential variation of the element too, so a linear
    field may be marked (Algorithm 10 tests every edge point), but limiting a
    linear field reproduces it: the minmod of equal differences is the exact
    slope.  With a TVB bound above every edge deviation nothing is marked."""
    cfg = _cfg(orc, p=p, pts=pts, bc_x=orc.TRANSMISSIVE, bc_y=orc.TRANSMISSIVE)
    x, y = orc.point_coords(cfg)
    q = np.stack([1.0 + 0.3 * x + 0.2 * y, 0.5 - 0.4 * x, 0.1 * y, 2.0 + 0.7 * x - 0.3 * y])
    ql, marks, margin, cnt = orc.limit(cfg, q)
    assert cnt > 0
    # boundary elements see a flat ghost average (transmissive) and are
    # flattened in that direction; interior elements are fixed points
    inner = np.zeros((cfg.ny, cfg.nx), bool)
    inner[1:-1, 1:-1] = True
    np.testing.assert_allclose(ql.reshape(4, cfg.ny, cfg.nx, -1)[:, inner],
                               q.reshape(4, cfg.ny, cfg.nx, -1)[:, inner], rtol=0, atol=1e-14)
    cfg.tvb_M = 1e3  # M h^2 = 15.6 / 36 > every |delta| here
    assert orc.limit(cfg, q)[3] == 0


@pytest.mark.parametrize("pts", [0, 1])
@pytest.mark.parametrize("p", [1, 2, 3])
def test_step_marks_and_monotone_limited_profile(orc, p, pts):
    nx, ny = 10, 3
    cfg = _cfg(orc, eqn=orc.ADVECTION, nx=nx, ny=ny, p=p, pts=pts, x1=1.0, y1=0.3,
               bc_x=orc.TRANSMISSIVE)
    x, y = orc.point_coords(cfg)
    step = 0.45  # inside element 4 (x in [0.4, 0.5])
    q = np.where(x >= step, 1.0, 0.0)[None]
    avg0 = orc.averages(cfg, q)
    ql, marks, margin, cnt = orc.limit(cfg, q)
    m2 = marks.reshape(ny, nx)
    expect = np.zeros((ny, nx), int)
    expect[:, 4] = 1
    np.testing.assert_array_equal(m2, expect)
    np.testing.assert_allclose(orc.averages(cfg, ql), avg0, rtol=0, atol=1e-15)
    n = p + 1
    rows = ql.reshape(ny, nx, n, n)  # [j, i, b, a]
    for j in range(ny):
        for b in range(n):
            prof = rows[j, :, b, :].ravel()
            assert np.all(np.diff(prof) >= -1e-15)
            assert prof.min() >= -1e-15 and prof.max() <= 1 + 1e-15
    # the limited element is linear with the minmod slope of its neighbours
    a4 = avg0[0].reshape(ny, nx)[:, 4]
    slope = np.minimum(1.0 - a4, a4 - 0.0) / 0.1
    xi = orc.tables(p, pts)["xi"]
    lim = a4[:, None] + (0.05 * xi)[None, :] * slope[:, None]
    np.testing.assert_allclose(rows[:, 4, 0, :], lim, rtol=0, atol=1e-14)


@pytest.mark.parametrize("pts", [0, 1])
@pytest.mark.parametrize("p", [1, 2, 3])
def test_step_in_y_with_unequal_spacing(orc, p, pts):
    """The same step along y on elements with hy = 2 hx: only the y slope is
    limited, scaled by hy."""
    nx, ny = 3, 10
    cfg = _cfg(orc, eqn=orc.ADVECTION, nx=nx, ny=ny, p=p, pts=pts, x1=0.3, y1=2.0,
               bc_y=orc.TRANSMISSIVE)
    x, y = orc.point_coords(cfg)
    # 0.3 below, 2.0 above, a 0 -> 1 step inside element row 4 (y in [0.8, 1.0]):
    # the backward difference of the averages is the smaller one
    row = (np.arange(nx * ny) // nx)[:, None] + 0 * y
    q = np.where(row < 4, 0.3, np.where(row > 4, 2.0, np.where(y >= 0.9, 1.0, 0.0)))[None]
    avg0 = orc.averages(cfg, q)
    ql, marks, _, _ = orc.limit(cfg, q)
    expect = np.zeros((ny, nx), int)
    expect[4, :] = 1
    np.testing.assert_array_equal(marks.reshape(ny, nx), expect)
    n = p + 1
    rows = ql.reshape(ny, nx, n, n)  # [j, i, b, a]
    a4 = avg0[0].reshape(ny, nx)[4, :]
    assert np.all(a4 - 0.3 < 2.0 - a4)
    slope = (a4 - 0.3) / 0.2
    xi = orc.tables(p, pts)["xi"]
    lim = a4[:, None] + (0.1 * xi)[None, :] * slope[:, None]   # [i, b]
    np.testing.assert_allclose(rows[4, :, :, 0], lim, rtol=0, atol=1e-14)
    np.testing.assert_allclose(orc.averages(cfg, ql), avg0, rtol=0, atol=1e-15)


def test_tvb_and_threshold(orc):
    cfg = _cfg(orc, eqn=orc.ADVECTION, nx=10, ny=2, p=2, x1=1.0, y1=0.2, bc_x=orc.TRANSMISSIVE)
    x, y = orc.point_coords(cfg)
    q = np.where(x >= 0.45, 1.0, 0.0)[None]
    assert orc.limit(cfg, q)[3] == 2
    cfg.tvb_M = 1e9  # |delta| <= M h^2 everywhere: TVB keeps every element
    assert orc.limit(cfg, q)[3] == 0
    cfg.tvb_M = 0.0
    # the same step scaled below the threshold is not marked, above it is
    assert orc.limit(cfg, 1e-4 * q)[3] == 0
    assert orc.limit(cfg, 1e-1 * q)[3] == 2
    _, _, margin, _ = orc.limit(cfg, 1e-1 * q)
    assert np.all(margin[np.array([4, 14])] > 0) and np.all(np.delete(margin, [4, 14]) < 0)


def test_limiter_keeps_averages_on_rough_states(orc):
    cfg = _cfg(orc, nx=9, ny=7, p=3)
    x, y = orc.point_coords(cfg)
    q = inputs.perturbed(inputs.vortex(x, y, eps=3.0, xc=0.5, yc=0.5, lx=1.0, ly=1.0), 11, 0.05)
    avg0 = orc.averages(cfg, q)
    ql, marks, _, cnt = orc.limit(cfg, q)
    assert cnt > 0
    assert not np.allclose(ql, q)
    np.testing.assert_allclose(orc.averages(cfg, ql), avg0, rtol=0, atol=1e-14)


# --------------------------------------------------------------------------
# adjoint
# --------------------------------------------------------------------------
def _rough_state(orc, cfg, seed):
    x, y = orc.point_coords(cfg)
    q = inputs.vortex(x, y, eps=3.0, xc=0.5 * (cfg.x0 + cfg.x1), yc=0.5 * (cfg.y0 + cfg.y1),
                      lx=cfg.x1 - cfg.x0, ly=cfg.y1 - cfg.y0)
    if cfg.eqn == orc.ADVECTION:
        q = q[:1]
    return inputs.perturbed(q, seed, 0.02)


@pytest.mark.parametrize("eqn", [0, 1])
@pytest.mark.parametrize("bc", [0, 1])
@pytest.mark.parametrize("p", [2, 3])
def test_residual_jvp_matches_central_differences(orc, eqn, bc, p):
    cfg = orc.Config(eqn=eqn, nx=4, ny=3, p=p, x1=2.0, y1=1.5, bc_x=bc, bc_y=bc,
                     flux=orc.RUSANOV, ax=0.8, ay=-0.5)
    q = _rough_state(orc, cfg, 5)
    rng = np.random.default_rng(9)
    for _ in range(3):
        v = rng.standard_normal(q.shape)
        h = 1e-6
        fd = (orc.residual(cfg, q + h * v) - orc.residual(cfg, q - h * v)) / (2 * h)
        jv = orc.residual_jvp(cfg, q, v)
        assert np.linalg.norm(fd - jv) <= 1e-7 * np.linalg.norm(jv)


@pytest.mark.parametrize("eqn", [0, 1])
@pytest.mark.parametrize("bc", [0, 1])
@pytest.mark.parametrize("p", [1, 2, 3])
def test_residual_vjp_dot_product(orc, eqn, bc, p):
    cfg = orc.Config(eqn=eqn, nx=4, ny=5, p=p, x1=2.0, y1=1.5, bc_x=bc, bc_y=1 - bc,
                     flux=orc.RUSANOV, ax=0.8, ay=-0.5)
    q = _rough_state(orc, cfg, 6)
    rng = np.random.default_rng(10)
    for _ in range(3):
        v = rng.standard_normal(q.shape)
        w = rng.standard_normal(q.shape)
        lhs = np.vdot(orc.residual_jvp(cfg, q, v), w)
        rhs = np.vdot(v, orc.residual_vjp(cfg, q, w))
        assert abs(lhs - rhs) <= 1e-13 * max(abs(lhs), 1.0) * 10


@pytest.mark.parametrize("eqn", [0, 1])
def test_rk3_vjp_matches_central_differences(orc, eqn):
    cfg = orc.Config(eqn=eqn, nx=4, ny=4, p=3, x1=2.0, y1=2.0, flux=orc.RUSANOV, ax=0.8, ay=-0.5)
    q = _rough_state(orc, cfg, 7)
    dt = 0.01
    rng = np.random.default_rng(11)
    for _ in range(3):
        v = rng.standard_normal(q.shape)
        w = rng.standard_normal(q.shape)
        h = 1e-6
        fd = (orc.rk3_step(cfg, q + h * v, dt) - orc.rk3_step(cfg, q - h * v, dt)) / (2 * h)
        lhs = np.vdot(fd, w)
        rhs = np.vdot(v, orc.rk3_vjp(cfg, q, dt, w))
        assert abs(lhs - rhs) <= 1e-7 * abs(rhs)
