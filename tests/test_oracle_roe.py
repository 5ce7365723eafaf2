"""Pins of the oracle's Roe flux (Roe's linearised Riemann solver with the
Harten-Hyman entropy fix): properties the solver has by construction,
checked on states built from closed forms."""
import math

import numpy as np
import pytest

import oracle

G = 1.4
NORMALS = [(1.0, 0.0), (0.0, 1.0), (-1.0, 0.0), (0.0, -1.0)]


def cfg(eqn=oracle.EULER, flux=oracle.ROE, **kw):
    return oracle.Config(eqn=eqn, flux=flux, gamma=G, **kw)


def cons(rho, u, v, p):
    return np.array([rho, rho * u, rho * v, p / (G - 1) + 0.5 * rho * (u * u + v * v)])


def euler_flux(q, nx, ny):
    """Eq. 4 along the normal, written out here."""
    rho, u, v = q[0], q[1] / q[0], q[2] / q[0]
    p = (G - 1) * (q[3] - 0.5 * rho * (u * u + v * v))
    vn = nx * u + ny * v
    return np.array([rho * vn, rho * u * vn + nx * p, rho * v * vn + ny * p, (q[3] + p) * vn])


def states(seed, n=20):
    rng = np.random.default_rng(seed)
    for _ in range(n):
        yield cons(rng.uniform(0.2, 3), rng.normal(0, 1.5), rng.normal(0, 1.5), rng.uniform(0.2, 4))


@pytest.mark.parametrize("nrm", NORMALS)
def test_consistency(nrm):
    c = cfg()
    for q in states(1):
        assert np.allclose(oracle.common_flux(c, q, q, *nrm), euler_flux(q, *nrm), rtol=1e-13, atol=1e-13)


def test_swap_symmetry():
    c = cfg()
    qs = list(states(2, 30))
    for a, b in zip(qs[::2], qs[1::2]):
        for nx, ny in NORMALS:
            Fab = oracle.common_flux(c, a, b, nx, ny)
            Fba = oracle.common_flux(c, b, a, -nx, -ny)
            assert np.allclose(Fab, -Fba, rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("nrm", NORMALS)
def test_stationary_contact_is_exact(nrm):
    """Equal pressure, zero normal velocity, any density and tangential
    velocity jump: the exact flux is the pressure alone."""
    c = cfg()
    nx, ny = nrm
    tx, ty = -ny, nx
    qm = cons(1.7, 0.8 * tx, 0.8 * ty, 2.2)
    qp = cons(0.4, -1.3 * tx, -1.3 * ty, 2.2)
    F = oracle.common_flux(c, qm, qp, nx, ny)
    assert np.allclose(F, [0.0, 2.2 * nx, 2.2 * ny, 0.0], rtol=0, atol=1e-13)


@pytest.mark.parametrize("mach", [1.5, 2.0, 4.0])
def test_stationary_normal_shock_is_exact(mach):
    """Rankine-Hugoniot states of a normal shock at rest (Mach `mach`
    upstream): Roe's linearisation resolves a single shock exactly, so the
    flux equals the (common) physical flux of both states."""
    c = cfg()
    rho1, p1 = 1.0, 1.0
    u1 = mach * math.sqrt(G * p1 / rho1)
    r = (G + 1) * mach ** 2 / ((G - 1) * mach ** 2 + 2)
    rho2, u2 = rho1 * r, u1 / r
    p2 = p1 * (1 + 2 * G / (G + 1) * (mach ** 2 - 1))
    qm, qp = cons(rho1, u1, 0.3, p1), cons(rho2, u2, 0.3, p2)
    F = oracle.common_flux(c, qm, qp, 1.0, 0.0)
    assert np.allclose(euler_flux(qm, 1, 0), euler_flux(qp, 1, 0), rtol=1e-12)
    assert np.allclose(F, euler_flux(qm, 1, 0), rtol=1e-12, atol=1e-12)


def test_supersonic_states_are_upwinded():
    """Both states faster than sound in +x: every wave moves the same way and
    the flux is the physical flux of the upstream state (the minus state for
    the normal +x, the plus state for the normal -x)."""
    c = cfg()
    qa = cons(1.0, 3.5, 0.2, 1.0)
    qb = cons(1.3, 3.2, -0.4, 1.4)
    assert np.allclose(oracle.common_flux(c, qa, qb, 1.0, 0.0), euler_flux(qa, 1, 0), rtol=1e-12)
    assert np.allclose(oracle.common_flux(c, qb, qa, -1.0, 0.0), euler_flux(qa, -1, 0), rtol=1e-12)


def test_advection_roe_is_upwind():
    cr, cu = cfg(oracle.ADVECTION, ax=0.7, ay=-1.1), cfg(oracle.ADVECTION, flux=oracle.UPWIND, ax=0.7, ay=-1.1)
    for nx, ny in NORMALS:
        a, b = np.array([0.3]), np.array([-1.4])
        assert np.allclose(oracle.common_flux(cr, a, b, nx, ny), oracle.common_flux(cu, a, b, nx, ny))


def test_roe_residual_preserves_freestream_and_conserves():
    o = oracle.Config(eqn=oracle.EULER, nx=10, ny=8, p=2, x1=10.0, y1=8.0, flux=oracle.ROE, cfl=0.08)
    x, y = oracle.point_coords(o)
    from paper_1709_01619_gb300 import inputs
    assert np.abs(oracle.residual(o, inputs.freestream(x))).max() <= 1e-12
    q = inputs.perturbed(inputs.vortex(x, y, eps=3.0, xc=5.0, yc=4.0, ly=8.0), 1, 0.02)
    s0 = oracle.averages(o, q).sum(axis=1)
    q1, _, _ = oracle.run(o, q, 10)
    assert np.allclose(oracle.averages(o, q1).sum(axis=1), s0, rtol=1e-13, atol=1e-12)


def test_roe_has_no_adjoint_in_the_oracle():
    o = oracle.Config(eqn=oracle.EULER, nx=4, ny=4, p=1, flux=oracle.ROE)
    q = np.ones(o.shape)
    with pytest.raises(ValueError):
        oracle.residual_vjp(o, q, q)
