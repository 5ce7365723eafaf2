"""Pins of the oracle's CPR residual, common flux and SSP-RK3.

Each test checks the oracle against something it does not compute itself:
an independent modal DG discretisation (FR with g_DG equals DG for a linear
flux), exact solutions and convergence orders, freestream preservation,
discrete conservation, the RK3 stability polynomial, the paper's printed
error tables, and the diagonal symmetry of the four-quadrant problem.
"""
import json
import math
import os

import numpy as np
import pytest
from numpy.polynomial import legendre as L

from paper_1709_01619_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def euler_flux(q, nx, ny, gamma=1.4):
    """Eq. 4, typed from the paper for the consistency check."""
    rho, mu, mv, e = q
    u, v = mu / rho, mv / rho
    p = (gamma - 1) * (e - 0.5 * rho * (u * u + v * v))
    f = np.array([mu, mu * u + p, mv * u, u * (e + p)])
    g = np.array([mv, mu * v, mv * v + p, v * (e + p)])
    return nx * f + ny * g


# --------------------------------------------------------------------------
# common flux
# --------------------------------------------------------------------------
def test_rusanov_consistency_and_conservation(orc):
    cfg = orc.Config(eqn=orc.EULER)
    rng = np.random.default_rng(3)
    for _ in range(20):
        prim = [rng.uniform(0.2, 2), rng.uniform(-1, 1), rng.uniform(-1, 1), rng.uniform(0.1, 2)]
        q = inputs.conserved(*prim)
        prim2 = [rng.uniform(0.2, 2), rng.uniform(-1, 1), rng.uniform(-1, 1), rng.uniform(0.1, 2)]
        q2 = inputs.conserved(*prim2)
        for nx, ny in ((1, 0), (0, 1), (0.6, 0.8)):
            F = orc.common_flux(cfg, q, q, nx, ny)
            np.testing.assert_allclose(F, euler_flux(q, nx, ny), rtol=1e-14, atol=1e-14)
            # flux through a face seen from the other side: F(a,b,n) = -F(b,a,-n)
            np.testing.assert_allclose(orc.common_flux(cfg, q, q2, nx, ny),
                                       -orc.common_flux(cfg, q2, q, -nx, -ny), rtol=1e-14, atol=1e-15)
        # Rusanov dissipation: lambda >= each one-sided speed, so F lies between
        # the central flux and the upwind-like jump term
        Fc = 0.5 * (euler_flux(q, 1, 0) + euler_flux(q2, 1, 0))
        d = orc.common_flux(cfg, q, q2, 1, 0) - Fc
        lam = -2 * d / (q2 - q)
        np.testing.assert_allclose(lam, lam[0], rtol=1e-9)
        c = lambda pr: math.sqrt(1.4 * pr[3] / pr[0])
        assert lam[0] == pytest.approx(max(abs(prim[1]) + c(prim), abs(prim2[1]) + c(prim2)), rel=1e-12)


def test_upwind_advection_flux(orc):
    for flux in (orc.UPWIND, orc.RUSANOV):
        cfg = orc.Config(eqn=orc.ADVECTION, ax=0.7, ay=-1.3, flux=flux)
        assert orc.common_flux(cfg, [2.0], [5.0], 1, 0)[0] == pytest.approx(0.7 * 2.0, rel=1e-15)
        assert orc.common_flux(cfg, [2.0], [5.0], 0, 1)[0] == pytest.approx(-1.3 * 5.0, rel=1e-15)


# --------------------------------------------------------------------------
# residual: equality with modal DG for linear advection
# --------------------------------------------------------------------------
def modal_dg_rhs(c, ax, ay, hx, hy):
    """Modal DG (Legendre basis, exact integrals, upwind flux) for
    u_t + ax u_x + ay u_y = 0 on a periodic grid.  c[j, i, m, k]: coefficient
    of P_m(xi) P_k(eta) in element (i, j).  Returns dc/dt."""
    ny, nx, n, _ = c.shape
    xg, wg = L.leggauss(n + 1)
    P = np.array([L.legval(xg, np.eye(n)[m]) for m in range(n)])            # P_m(x_g)
    dP = np.array([L.legval(xg, L.legder(np.eye(n)[m])) for m in range(n)])  # P_m'(x_g)
    K = np.einsum("g,mg,kg->mk", wg, dP, P)                                   # int P_k P_m'
    p1 = np.ones(n)                                                           # P_m(1)
    m1 = (-1.0) ** np.arange(n)                                               # P_m(-1)
    inv_mass = (2 * np.arange(n) + 1) / 2.0
    out = np.zeros_like(c)
    # x direction, per eta mode k: trace u(+-1) = sum_j c_jk P_j(+-1)
    tr_r = np.einsum("yxmk,m->yxk", c, p1)
    tr_l = np.einsum("yxmk,m->yxk", c, m1)
    up_r = ax * (tr_r if ax >= 0 else np.roll(tr_l, -1, axis=1))   # flux at right face
    up_l = np.roll(up_r, 1, axis=1)                                 # flux at left face
    vol = ax * np.einsum("mj,yxjk->yxmk", K, c)
    out += (2 / hx) * inv_mass[None, None, :, None] * (
        vol - p1[None, None, :, None] * up_r[:, :, None, :] + m1[None, None, :, None] * up_l[:, :, None, :])
    tr_t = np.einsum("yxkm,m->yxk", c, p1)
    tr_b = np.einsum("yxkm,m->yxk", c, m1)
    up_t = ay * (tr_t if ay >= 0 else np.roll(tr_b, -1, axis=0))
    up_b = np.roll(up_t, 1, axis=0)
    vol = ay * np.einsum("mj,yxkj->yxkm", K, c)
    out += (2 / hy) * inv_mass[None, None, None, :] * (
        vol - p1[None, None, None, :] * up_t[:, :, :, None] + m1[None, None, None, :] * up_b[:, :, :, None])
    return out


@pytest.mark.parametrize("pts", [0, 1])
@pytest.mark.parametrize("p", [1, 2, 3, 4])
@pytest.mark.parametrize("a", [(1.0, 0.6), (-0.8, 1.7)])
def test_advection_residual_equals_modal_dg(orc, p, pts, a):
    nx, ny, n = 5, 4, p + 1
    cfg = orc.Config(eqn=orc.ADVECTION, nx=nx, ny=ny, p=p, pts=pts, flux=orc.UPWIND,
                     ax=a[0], ay=a[1], x1=1.25, y1=0.8)
    rng = np.random.default_rng(100 + p)
    c = rng.standard_normal((ny, nx, n, n))
    xi = orc.tables(p, pts)["xi"]
    V = np.array([L.legval(xi, np.eye(n)[m]) for m in range(n)]).T  # V[a, m] = P_m(xi_a)
    # nodal values q[e, b*n + a] = sum_{m,k} c[m,k] P_m(xi_a) P_k(eta_b)
    q = np.einsum("am,bk,yxmk->yxba", V, V, c).reshape(1, nx * ny, n * n)
    R = orc.residual(cfg, q)
    dc = modal_dg_rhs(c, a[0], a[1], 1.25 / nx, 0.8 / ny)
    Rdg = np.einsum("am,bk,yxmk->yxba", V, V, dc).reshape(1, nx * ny, n * n)
    scale = np.abs(Rdg).max()
    np.testing.assert_allclose(R, Rdg, rtol=0, atol=2e-13 * scale)
    cfg.flux = orc.RUSANOV
    np.testing.assert_allclose(orc.residual(cfg, q), Rdg, rtol=0, atol=2e-13 * scale)


# --------------------------------------------------------------------------
# residual: exact solutions, freestream, conservation
# --------------------------------------------------------------------------
@pytest.mark.parametrize("p,grids", [(1, (8, 16, 32)), (2, (6, 12, 24)), (3, (4, 8, 16))])
def test_advection_convergence_order(orc, p, grids):
    """L2 error of the point values vs sin(2 pi (x - t)) sin(2 pi (y - t))
    falls at least like h^(p+1) (time step small enough not to matter)."""
    errs = []
    T = 0.1
    for N in grids:
        cfg = orc.Config(eqn=orc.ADVECTION, nx=N, ny=N, p=p, flux=orc.UPWIND, ax=1.0, ay=1.0)
        x, y = orc.point_coords(cfg)
        q = inputs.advection_sine(x, y)
        dt0 = 0.005 / N
        ns = int(math.ceil(T / dt0))
        qT, _, _ = orc.run(cfg, q, ns, T / ns)
        errs.append(np.sqrt(np.mean((qT[0] - inputs.advection_sine(x - T, y - T)[0]) ** 2)))
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert rates.min() > p + 1 - 0.25, (errs, rates)


@pytest.mark.parametrize("pts", [0, 1])
@pytest.mark.parametrize("div", [0, 1])
@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_freestream_preservation(orc, p, pts, div):
    for bc in (orc.PERIODIC, orc.TRANSMISSIVE):
        cfg = orc.Config(eqn=orc.EULER, nx=5, ny=3, p=p, pts=pts, div=div, x1=2.0, y1=0.9,
                         bc_x=bc, bc_y=bc)
        x, y = orc.point_coords(cfg)
        R = orc.residual(cfg, inputs.freestream(x))
        assert np.abs(R).max() < 1e-12


def test_conservation_periodic_euler(orc):
    cfg = orc.Config(eqn=orc.EULER, nx=8, ny=8, p=3, x1=10, y1=10, cfl=0.08)
    x, y = orc.point_coords(cfg)
    q = inputs.vortex(x, y, eps=5.0)
    s0 = orc.norms(cfg, q)["sum_avg"]
    qT, n, _ = orc.run(cfg, q, 40)
    s1 = orc.norms(cfg, qT)["sum_avg"]
    assert n == 40
    np.testing.assert_allclose(s1, s0, rtol=2e-14, atol=1e-13)
    assert not np.allclose(qT, q)


def test_conservation_with_limiter(orc):
    cfg = orc.Config(eqn=orc.EULER, nx=12, ny=12, p=2, x0=-1, x1=1, y0=-1, y1=1, cfl=0.1,
                     limiter=1, tvb_M=50.0, lim_eps=1e-3)
    x, y = orc.point_coords(cfg)
    q = inputs.radial_shock(x, y)
    s0 = orc.norms(cfg, q)["sum_avg"]
    qT, _, _ = orc.run(cfg, q, 10)
    np.testing.assert_allclose(orc.norms(cfg, qT)["sum_avg"], s0, rtol=1e-13, atol=1e-13)
    assert orc.norms(cfg, qT)["n_nonphys"] == 0


def test_conservation_over_a_thousand_limited_steps(orc):
    """Periodic LP CPR with the limiter acting after every stage: the sum of
    the element averages, formed here with numpy's Gauss weights from the
    point values (not by the oracle), stays constant over 1000 SSP-RK3 steps
    while the waves of a discontinuous start cross the periodic boundaries.
    M = 0 (plain minmod test): on a grid this coarse the TVB bound M h^2
    with the workload's M = 50 would exceed every jump and switch the
    limiter off, and the unlimited scheme loses positivity."""
    p = 2
    cfg = orc.Config(eqn=orc.EULER, nx=10, ny=10, p=p, x0=-1, x1=1, y0=-1, y1=1, cfl=0.1,
                     limiter=1, tvb_M=0.0, lim_eps=1e-3)
    x, y = orc.point_coords(cfg)
    q = np.asarray(inputs.radial_shock(x, y), dtype=np.float64).reshape(cfg.shape)
    _, w = np.polynomial.legendre.leggauss(p + 1)
    W = np.outer(w, w).ravel() / 4.0  # point b*n + a gets w_b w_a / 4

    def total(state):
        return (np.asarray(state).reshape(cfg.shape) * W).sum(axis=(1, 2))

    s0 = total(q)
    _, marks0, _, _ = orc.limit(cfg, q)
    qT, n, t = orc.run(cfg, q, 1000)
    assert n == 1000 and t > 1.0  # long enough for the waves to wrap around
    # round-off only: about 1e-16 per point and stage, summed as a random walk
    # over 900 points and 3000 stages gives ~2e-13
    np.testing.assert_allclose(total(qT), s0, rtol=1e-12, atol=1e-12)
    assert marks0.sum() > 0
    assert orc.norms(cfg, qT)["n_nonphys"] == 0


def test_rk3_is_third_order_taylor_polynomial(orc):
    """For the linear advection operator R(q) = A q, one SSP-RK3 step must equal
    (I + dt A + dt^2 A^2 / 2 + dt^3 A^3 / 6) q."""
    cfg = orc.Config(eqn=orc.ADVECTION, nx=4, ny=3, p=2, ax=0.9, ay=-0.4, flux=orc.UPWIND)
    q = np.random.default_rng(7).standard_normal(cfg.shape)
    dt = 0.013
    A1 = orc.residual(cfg, q)
    A2 = orc.residual(cfg, A1)
    A3 = orc.residual(cfg, A2)
    expect = q + dt * A1 + dt ** 2 / 2 * A2 + dt ** 3 / 6 * A3
    np.testing.assert_allclose(orc.rk3_step(cfg, q, dt), expect, rtol=0, atol=1e-13)


def test_dt_formula_freestream(orc):
    cfg = orc.Config(eqn=orc.EULER, nx=4, ny=5, p=2, x1=2.0, y1=2.0, cfl=0.3)
    x, _ = orc.point_coords(cfg)
    q = inputs.freestream(x, rho=1.2, u=0.5, v=-1.2, p=0.8)
    speed = math.hypot(0.5, 1.2) + math.sqrt(1.4 * 0.8 / 1.2)
    assert orc.max_wave(cfg, q) == pytest.approx(speed, rel=1e-14)
    assert orc.dt(cfg, q) == pytest.approx(0.3 * 0.4 / speed, rel=1e-14)


def test_max_wave_is_the_maximum_over_every_solution_point(orc):
    """The CFL speed (Eq. 36) is the largest |V| + c over all solution
    points, not over element averages: a brute-force maximum over the state
    array, with one point of one element made the fastest."""
    cfg = orc.Config(eqn=orc.EULER, nx=5, ny=4, p=3, x1=2.5, y1=2.0, cfl=0.2)
    x, y = orc.point_coords(cfg)
    q = inputs.perturbed(inputs.vortex(x, y, eps=2.0, xc=1.25, yc=1.0, lx=2.5, ly=2.0), 11, 0.02)
    q = np.array(q, dtype=np.float64).reshape(cfg.shape)
    # one point of one element set to a fast state (rho, u, v, p) = (1, 4, 0.3, 1)
    q[:, 13, 6] = [1.0, 4.0, 0.3, 1.0 / 0.4 + 0.5 * (16.0 + 0.09)]
    rho, mx, my, E = q
    u, v = mx / rho, my / rho
    p = 0.4 * (E - 0.5 * rho * (u * u + v * v))
    brute = np.max(np.sqrt(u * u + v * v) + np.sqrt(1.4 * p / rho))
    assert np.argmax(np.sqrt(u * u + v * v) + np.sqrt(1.4 * p / rho)) == 13 * 16 + 6
    assert orc.max_wave(cfg, q) == pytest.approx(brute, rel=1e-14)
    assert orc.dt(cfg, q) == pytest.approx(0.2 * 0.5 / brute, rel=1e-14)


# --------------------------------------------------------------------------
# the paper's tables (loose pins; see the readings in the design notes)
# --------------------------------------------------------------------------
def _paper_vortex_errors(orc, p, grids, cfls):
    errs = []
    for N, cfl in zip(grids, cfls):
        cfg = orc.Config(eqn=orc.EULER, nx=N, ny=N, p=p, x0=-5, x1=5, y0=-5, y1=5,
                         pts=orc.LOBATTO, div=orc.DIV_CHAIN, cfl=cfl)
        x, y = orc.point_coords(cfg)
        q = inputs.vortex(x, y, eps=5.0, xc=0.0, yc=0.0, uinf=1.0, vinf=0.0)
        qT, _, t = orc.run(cfg, q, 100000, 0.0, 1.0)
        assert t == pytest.approx(1.0, abs=1e-12)
        ex = orc.exact_averages(cfg, "vortex", 1.0, [5.0, 0.0, 0.0, 1.0, 0.0])
        errs.append(orc.rho_avg_error(cfg, qT, ex))
    return np.array(errs)


def test_table6_p1_slopes_and_magnitude(orc):
    """Paper settings (Lobatto points, chain-rule divergence, Rusanov, CFL 0.24):
    the printed P1 slopes are reproduced to 0.05 and the errors to a factor 1.5."""
    with open(os.path.join(GOLDEN, "paper_tables_6_7.json")) as f:
        gold = json.load(f)
    grids = gold["grids"]
    e = _paper_vortex_errors(orc, 1, grids, gold["cfl_p1"])
    slopes = np.log(e[:-1] / e[1:]) / np.log(np.array(grids[1:]) / np.array(grids[:-1]))
    np.testing.assert_allclose(slopes, gold["cpr_p1_slope"][1:], atol=0.05)
    ratio = e / np.array(gold["cpr_p1_error"])
    assert np.all((ratio > 1 / 1.5) & (ratio < 1.5)), ratio


def test_table7_p2_bounded_by_paper(orc):
    """P2: the oracle's errors stay below the printed ones and fall at least
    as fast as the printed slopes (the printed P2 values carry an additional
    error source the paper does not identify)."""
    with open(os.path.join(GOLDEN, "paper_tables_6_7.json")) as f:
        gold = json.load(f)
    grids = gold["grids"][:3]
    e = _paper_vortex_errors(orc, 2, grids, gold["cfl_p2"][:3])
    assert np.all(e < np.array(gold["cpr_p2_error"][:3]))
    assert np.all(e > 0.05 * np.array(gold["cpr_p2_error"][:3]))
    slopes = np.log(e[:-1] / e[1:]) / np.log(np.array(grids[1:]) / np.array(grids[:-1]))
    assert np.all(slopes >= np.array(gold["cpr_p2_slope"][1:3]))


# --------------------------------------------------------------------------
# four-quadrant problem: diagonal symmetry and positivity
# --------------------------------------------------------------------------
def test_four_quadrant_diagonal_symmetry(orc):
    N, p = 16, 2
    cfg = orc.Config(eqn=orc.EULER, nx=N, ny=N, p=p, bc_x=orc.TRANSMISSIVE, bc_y=orc.TRANSMISSIVE,
                     limiter=1, tvb_M=50.0, lim_eps=1e-3, cfl=0.1)
    x, y = orc.point_coords(cfg)
    q = inputs.four_quadrant(x, y)
    _, marks0, _, _ = orc.limit(cfg, q)
    qT, _, _ = orc.run(cfg, q, 8)
    n = p + 1
    A = qT.reshape(4, N, N, n, n)                       # [v, j, i, b, a]
    M = A.transpose(0, 2, 1, 4, 3)[[0, 2, 1, 3]]        # mirror x<->y, swap momenta
    np.testing.assert_allclose(A, M, rtol=0, atol=1e-12)
    nrm = orc.norms(cfg, qT)
    assert nrm["n_nonphys"] == 0
    assert marks0.sum() > 0
