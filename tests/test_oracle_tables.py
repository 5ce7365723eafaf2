"""Pins of the oracle's 1D operator tables against closed forms and numpy.

None of these re-derives a table the way the oracle does (Newton iteration on
Legendre polynomials, product formulas for the Lagrange basis): they check
the tables against textbook closed forms, numpy's Legendre routines and the
polynomial identities that define each table.
"""
import json
import math
import os

import numpy as np
import pytest
from numpy.polynomial import legendre as L

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _ev(s):
    return float(eval(s, {"sqrt": math.sqrt}))


@pytest.mark.parametrize("kind", ["gauss", "lobatto"])
def test_nodes_weights_closed_forms(orc, kind):
    with open(os.path.join(GOLDEN, "quadrature_closed_forms.json")) as f:
        gold = json.load(f)[kind]
    pts = orc.GAUSS if kind == "gauss" else orc.LOBATTO
    for n_str, rule in gold.items():
        n = int(n_str)
        t = orc.tables(n - 1, pts)
        np.testing.assert_allclose(t["xi"], [_ev(s) for s in rule["nodes"]], rtol=0, atol=2e-16 * 4)
        np.testing.assert_allclose(t["w"], [_ev(s) for s in rule["weights"]], rtol=0, atol=4e-16 * 4)


@pytest.mark.parametrize("n", range(2, 8))
def test_gauss_matches_numpy(orc, n):
    x, w = L.leggauss(n)
    t = orc.tables(n - 1, orc.GAUSS)
    np.testing.assert_allclose(t["xi"], x, rtol=0, atol=1e-15)
    np.testing.assert_allclose(t["w"], w, rtol=0, atol=1e-15)


@pytest.mark.parametrize("p", range(1, 7))
def test_lobatto_interior_roots_of_dPp(orc, p):
    t = orc.tables(p, orc.LOBATTO)
    roots = np.sort(np.real(L.Legendre.basis(p).deriv().roots()))
    np.testing.assert_allclose(t["xi"][1:-1], roots, rtol=0, atol=1e-14)
    assert t["xi"][0] == -1.0 and t["xi"][-1] == 1.0
    # weights integrate polynomials up to degree 2p - 1 exactly
    for m in range(2 * p):
        exact = (1 - (-1) ** (m + 1)) / (m + 1)
        assert abs(np.dot(t["w"], t["xi"] ** m) - exact) < 1e-14


@pytest.mark.parametrize("pts", [0, 1])
@pytest.mark.parametrize("p", range(1, 7))
def test_derivative_and_edge_tables_exact_on_monomials(orc, p, pts):
    t = orc.tables(p, pts)
    xi = t["xi"]
    for m in range(p + 1):
        # D differentiates every degree-p polynomial exactly
        d = t["D"] @ (xi ** m)
        exact = m * xi ** (m - 1) if m > 0 else np.zeros_like(xi)
        np.testing.assert_allclose(d, exact, rtol=0, atol=1e-12 * (1 + m * m))
        # edge interpolation is exact
        assert abs(np.dot(t["lm"], xi ** m) - (-1.0) ** m) < 1e-13
        assert abs(np.dot(t["lp"], xi ** m) - 1.0) < 1e-13
    # rows of D sum to zero (derivative of a constant)
    np.testing.assert_allclose(t["D"].sum(axis=1), 0.0, atol=1e-12)


@pytest.mark.parametrize("pts", [0, 1])
@pytest.mark.parametrize("p", range(1, 7))
def test_radau_correction_derivatives(orc, p, pts):
    """g_L, g_R are the right/left Radau polynomials of degree p+1 (g_DG).

    Checked against numpy's Legendre derivative of the closed form, the end
    values through quadrature (integral of g' = jump of g), and the lifting
    identity int g_L' phi = -phi(-1) for phi of degree < p that follows from
    the Radau orthogonality (this is what makes FR with g_DG equal to DG)."""
    t = orc.tables(p, pts)
    xi, w = t["xi"], t["w"]
    cL = np.zeros(p + 2)
    cL[p + 1], cL[p] = 1.0, -1.0
    cL *= 0.5 * (-1.0) ** (p + 1)
    cR = np.zeros(p + 2)
    cR[p + 1], cR[p] = 0.5, 0.5
    np.testing.assert_allclose(t["dgl"], L.legval(xi, L.legder(cL)), rtol=0, atol=1e-12)
    np.testing.assert_allclose(t["dgr"], L.legval(xi, L.legder(cR)), rtol=0, atol=1e-12)
    assert abs(L.legval(-1.0, cL) - 1.0) < 1e-14 and abs(L.legval(1.0, cL)) < 1e-14
    assert abs(L.legval(1.0, cR) - 1.0) < 1e-14 and abs(L.legval(-1.0, cR)) < 1e-14
    assert abs(np.dot(w, t["dgl"]) + 1.0) < 1e-13
    assert abs(np.dot(w, t["dgr"]) - 1.0) < 1e-13
    for m in range(p):
        assert abs(np.dot(w, t["dgl"] * xi ** m) + (-1.0) ** m) < 1e-12
        assert abs(np.dot(w, t["dgr"] * xi ** m) - 1.0) < 1e-12


def test_legendre_values(orc):
    x = np.linspace(-1, 1, 9)
    for k in range(8):
        c = np.zeros(k + 1)
        c[k] = 1
        np.testing.assert_allclose([orc.legendre(k, v) for v in x], L.legval(x, c), atol=1e-14)
        np.testing.assert_allclose([orc.legendre_d(k, v) for v in x],
                                   L.legval(x, L.legder(c)), atol=1e-12)
