"""Pins of the oracle's nodal-DG edge correction (Sec. 2.3): the lifting
operator L = M^-1 M^A of the strong form, with the exact mass matrix
(OR_CORR_NDG) or with the integrals taken by the solution points' own
quadrature (OR_CORR_NDG_LUMPED).

Each check follows from the mathematics, not from the oracle's formulas:
the equivalence of DG with FR/CPR using the Radau correction g_DG (Huynh),
exactness of the n-point Gauss rule for degree 2p, the Gauss-Lobatto end
weight 2/(p(p+1)), and the 2D lifting matrix assembled here by brute force
from the tensor-product basis."""
import numpy as np
import pytest

import oracle
from paper_1709_01619_gb300 import inputs

ORDERS = [1, 2, 3, 4]


def lag(xi, i, x):
    r = np.ones_like(np.asarray(x, dtype=float))
    for m in range(len(xi)):
        if m != i:
            r = r * (x - xi[m]) / (xi[i] - xi[m])
    return r


@pytest.mark.parametrize("pts", [oracle.GAUSS, oracle.LOBATTO])
@pytest.mark.parametrize("p", ORDERS)
def test_exact_lift_equals_radau_derivatives(p, pts):
    """DG with the exact mass matrix and CPR with g_DG are the same scheme, so
    M^-1 l(+1) = g_R'(xi) and -M^-1 l(-1) = g_L'(xi) at every point."""
    a = oracle.tables(p, pts)
    b = oracle.tables(p, pts, oracle.CORR_NDG)
    assert np.abs(a["dgr"] - b["dgr"]).max() <= 1e-12
    assert np.abs(a["dgl"] - b["dgl"]).max() <= 1e-12


@pytest.mark.parametrize("p", ORDERS)
def test_lumped_equals_exact_on_gauss_points(p):
    """The n-point Gauss rule integrates the degree-2p products l_i l_j
    exactly, so the lumped mass matrix is the exact one."""
    a = oracle.tables(p, oracle.GAUSS, oracle.CORR_NDG)
    b = oracle.tables(p, oracle.GAUSS, oracle.CORR_NDG_LUMPED)
    assert np.abs(a["dgr"] - b["dgr"]).max() <= 1e-12
    assert np.abs(a["dgl"] - b["dgl"]).max() <= 1e-12


@pytest.mark.parametrize("p", ORDERS)
def test_lumped_lobatto_lift_acts_on_the_end_node_only(p):
    """With Gauss-Lobatto points l_a(+1) is 1 at the last node and 0
    elsewhere, and the end weight is 2/(p(p+1)): the lumped lift is
    p(p+1)/2 at the end node.  It differs from the exact (Radau) one."""
    t = oracle.tables(p, oracle.LOBATTO, oracle.CORR_NDG_LUMPED)
    k = p * (p + 1) / 2.0
    assert np.allclose(t["dgr"], [0.0] * p + [k], rtol=0, atol=1e-12)
    assert np.allclose(t["dgl"], [-k] + [0.0] * p, rtol=0, atol=1e-12)
    r = oracle.tables(p, oracle.LOBATTO)
    assert np.abs(t["dgr"] - r["dgr"]).max() > 0.1


@pytest.mark.parametrize("corr", [oracle.CORR_NDG, oracle.CORR_NDG_LUMPED])
@pytest.mark.parametrize("pts", [oracle.GAUSS, oracle.LOBATTO])
def test_each_lift_integrates_to_one(corr, pts):
    """sum_a w_a g_R'(xi_a) = g_R(1) - g_R(-1) = 1: the discrete statement
    that the correction moves the edge flux jump into the element exactly
    once (what makes the averages conservative)."""
    for p in ORDERS:
        t = oracle.tables(p, pts, corr)
        assert abs((t["w"] * t["dgr"]).sum() - 1.0) <= 1e-13
        assert abs((t["w"] * t["dgl"]).sum() + 1.0) <= 1e-13


@pytest.mark.parametrize("pts", [oracle.GAUSS, oracle.LOBATTO])
@pytest.mark.parametrize("p", [1, 2, 3])
def test_2d_lifting_matrix_by_brute_force(p, pts):
    """Assemble the 2D mass matrix M_2d = int l_a(xi) l_b(eta) l_a'(xi)
    l_b'(eta) and the face mass matrix of the face xi = +1,
    M^A[(a,b), c] = int l_a(1) l_b(eta) l_c(eta) d eta, with a Gauss rule of
    n + 1 points per direction (numpy), and check L = M_2d^-1 M^A against the
    oracle's line lift: L[(a,b), c] = dgr[a] * delta_bc."""
    n = p + 1
    xi = oracle.tables(p, pts)["xi"]
    gx, gw = np.polynomial.legendre.leggauss(n + 1)
    B = np.array([lag(xi, i, gx) for i in range(n)])          # B[i, q] = l_i(x_q)
    M1 = (B * gw) @ B.T
    M2 = np.kron(M1, M1)                                       # index b*n + a (eta slow)
    l1 = np.array([lag(xi, i, 1.0) for i in range(n)])
    MA = np.zeros((n * n, n))
    for b in range(n):
        for a in range(n):
            for c in range(n):
                MA[b * n + a, c] = l1[a] * M1[b, c]
    L = np.linalg.solve(M2, MA)
    dgr = oracle.tables(p, pts, oracle.CORR_NDG)["dgr"]
    expect = np.zeros((n * n, n))
    for b in range(n):
        for a in range(n):
            expect[b * n + a, b] = dgr[a]
    assert np.abs(L - expect).max() <= 1e-11


@pytest.mark.parametrize("div", [oracle.DIV_LP, oracle.DIV_CHAIN])
@pytest.mark.parametrize("pts", [oracle.GAUSS, oracle.LOBATTO])
def test_ndg_residual_equals_cpr_residual(pts, div):
    for p in ORDERS:
        kw = dict(eqn=oracle.EULER, nx=7, ny=6, p=p, pts=pts, div=div, x1=3.5, y1=3.0)
        cg = oracle.Config(**kw)
        cn = oracle.Config(corr=oracle.CORR_NDG, **kw)
        x, y = oracle.point_coords(cg)
        q = inputs.perturbed(inputs.vortex(x, y, eps=3.0, xc=1.75, yc=1.5, lx=3.5, ly=3.0), p, 0.02)
        Rg, Rn = oracle.residual(cg, q), oracle.residual(cn, q)
        assert np.linalg.norm(Rn - Rg) <= 1e-12 * np.linalg.norm(Rg)


def test_lumped_lobatto_conserves_averages():
    c = oracle.Config(eqn=oracle.EULER, nx=10, ny=8, p=3, pts=oracle.LOBATTO, corr=oracle.CORR_NDG_LUMPED,
                      x1=10.0, y1=8.0, cfl=0.05)
    x, y = oracle.point_coords(c)
    q = inputs.perturbed(inputs.vortex(x, y, eps=3.0, xc=5.0, yc=4.0, ly=8.0), 2, 0.02)
    s0 = oracle.averages(c, q).sum(axis=1)
    q1, _, _ = oracle.run(c, q, 15)
    assert np.allclose(oracle.averages(c, q1).sum(axis=1), s0, rtol=1e-13, atol=1e-12)


@pytest.mark.parametrize("p", [2, 3])
def test_lumped_lobatto_converges_on_advection(p):
    """Linear advection of sin(2 pi x) sin(2 pi y) on the unit square to
    t = 0.05 with upwind fluxes: the L2 error of the point values falls at
    order >= p + 1/2 over 8, 16, 32 elements per direction."""
    errs = []
    for n in (8, 16, 32):
        c = oracle.Config(eqn=oracle.ADVECTION, nx=n, ny=n, p=p, pts=oracle.LOBATTO,
                          corr=oracle.CORR_NDG_LUMPED, flux=oracle.UPWIND, ax=1.0, ay=1.0)
        x, y = oracle.point_coords(c)
        q0 = (np.sin(2 * np.pi * x) * np.sin(2 * np.pi * y))[None]
        t = 0.05
        nst = int(np.ceil(t / (0.02 / n)))
        q, _, _ = oracle.run(c, q0, nst, t / nst)
        ex = np.sin(2 * np.pi * (x - t)) * np.sin(2 * np.pi * (y - t))
        errs.append(np.sqrt(np.mean((q[0] - ex) ** 2)))
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert rates.min() >= p + 0.5, (errs, rates)
