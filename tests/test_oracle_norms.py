"""Pins of the oracle's norms (the FP64 reductions of the hot path: the sums of
element averages of Algorithm 9, the L2 error against a reference, the
largest signal speed of Eq. 36 and the count of non-physical points), each
against something other than the oracle itself: numpy's norm, closed-form
integrals of polynomials that the solution points' quadrature integrates
exactly, brute-force maxima, and points planted to be non-physical."""
import numpy as np
import pytest

import oracle as orc


def cfg(eqn=orc.EULER, nx=5, ny=4, p=2, **kw):
    return orc.Config(eqn=eqn, nx=nx, ny=ny, p=p, x0=0.0, x1=2.0, y0=0.0, y1=3.0, **kw)


def smooth_state(c, seed=0):
    x, y = orc.point_coords(c)
    rng = np.random.default_rng(seed)
    if c.eqn == orc.ADVECTION:
        return (np.sin(x) * np.cos(y) + 0.1 * rng.standard_normal(x.shape))[None]
    rho = 1.0 + 0.2 * np.sin(x + y)
    u, v = 0.3 * np.cos(y), -0.2 * np.sin(x)
    p = 1.0 + 0.1 * np.cos(x * y)
    return np.stack([rho, rho * u, rho * v, p / 0.4 + 0.5 * rho * (u * u + v * v)])


@pytest.mark.parametrize("eqn", [orc.ADVECTION, orc.EULER])
def test_l2_matches_numpy_norm(eqn):
    c = cfg(eqn)
    q, ref = smooth_state(c, 1), smooth_state(c, 2)
    n = orc.norms(c, q, ref)
    d = np.linalg.norm((q - ref).ravel())
    assert n["l2_abs"] == pytest.approx(d, rel=1e-13)
    assert n["l2_rel"] == pytest.approx(d / np.linalg.norm(ref.ravel()), rel=1e-13)


def test_l2_of_a_constant_offset_is_closed_form():
    """q = ref + c at every one of the V * npts values: ||q - ref|| =
    |c| sqrt(V * npts); a zero reference gives l2_rel = l2_abs."""
    c = cfg(orc.EULER, nx=3, ny=7, p=3)
    ref = smooth_state(c, 3)
    n = orc.norms(c, ref + 0.25, ref)
    count = ref.size
    assert n["l2_abs"] == pytest.approx(0.25 * np.sqrt(count), rel=1e-13)
    z = orc.norms(c, ref, np.zeros_like(ref))
    assert z["l2_rel"] == z["l2_abs"] == pytest.approx(np.linalg.norm(ref.ravel()), rel=1e-13)
    assert orc.norms(c, ref)["l2_abs"] == 0.0  # no reference given


@pytest.mark.parametrize("pts", [orc.GAUSS, orc.LOBATTO])
@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_sum_of_averages_is_the_integral(p, pts):
    """For fields of degree <= p in each coordinate the element averages are
    exact (the point rule integrates degree 2p-1 or more), so the sum over
    elements equals (1 / (hx hy)) times the integral over the domain."""
    c = cfg(orc.EULER, nx=5, ny=4, p=p, pts=pts)
    x, y = orc.point_coords(c)
    hx, hy = 2.0 / 5, 3.0 / 4
    fields = [x ** p * y, 1.0 + 0 * x, x * y ** p, 2.0 - y]
    exact = [(2.0 ** (p + 1) / (p + 1)) * (9.0 / 2), 6.0, 2.0 * 3.0 ** (p + 1) / (p + 1), 12.0 - 9.0]
    q = np.stack(fields)
    n = orc.norms(c, q)
    np.testing.assert_allclose(n["sum_avg"], np.array(exact) / (hx * hy), rtol=1e-13)


def test_max_wave_is_the_brute_force_maximum():
    c = cfg(orc.EULER, nx=4, ny=3, p=3)
    q = smooth_state(c, 4)
    rho, u, v = q[0], q[1] / q[0], q[2] / q[0]
    p = 0.4 * (q[3] - 0.5 * rho * (u * u + v * v))
    speed = np.sqrt(u * u + v * v) + np.sqrt(1.4 * p / rho)
    assert orc.norms(c, q)["max_wave"] == pytest.approx(speed.max(), rel=1e-14)


def test_nonphysical_points_are_counted_once_each():
    """Planted: negative density; zero energy with zero momentum (pressure 0,
    not > 0); a NaN momentum; an infinite energy; and one point that is bad
    twice over (negative density and NaN), which counts once."""
    c = cfg(orc.EULER, nx=4, ny=4, p=2)
    q = smooth_state(c, 5).copy()
    assert orc.norms(c, q)["n_nonphys"] == 0
    q[0, 1, 2] = -0.5
    q[1, 3, 0] = q[2, 3, 0] = q[3, 3, 0] = 0.0
    q[2, 5, 4] = np.nan
    q[3, 7, 8] = np.inf
    q[0, 9, 1] = -1.0
    q[1, 9, 1] = np.nan
    n = orc.norms(c, q)
    assert n["n_nonphys"] == 5
    assert n["max_wave"] < 0  # no speed is reported for a state with bad points


def test_nonphysical_count_for_advection_is_non_finite_only():
    c = cfg(orc.ADVECTION, nx=3, ny=3, p=1)
    q = -np.abs(smooth_state(c, 6))  # negative values are physical here
    assert orc.norms(c, q)["n_nonphys"] == 0
    q[0, 2, 1] = np.nan
    q[0, 4, 3] = -np.inf
    assert orc.norms(c, q)["n_nonphys"] == 2
