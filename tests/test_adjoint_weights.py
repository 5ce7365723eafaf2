"""The misfit weights of the adjoint workload (host code, no GPU): they are
the quadrature of the configuration's own solution points, so that the
weighted sum of a polynomial field integrates it."""
import types

import numpy as np
import pytest

import oracle
from paper_1709_01619_gb300 import _native as nat
from paper_1709_01619_gb300 import adjoint


@pytest.mark.parametrize("pts", [nat.GAUSS, nat.LOBATTO])
@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_weights_are_the_solution_points_quadrature(p, pts):
    n = p + 1
    w = adjoint.point_weights(n, pts == nat.LOBATTO)
    t = oracle.tables(p, pts)
    assert np.allclose(w, t["w"], rtol=0, atol=1e-13)
    # the rule integrates x^m on [-1, 1] for m up to 2n - 1 (Gauss) or 2n - 3 (Lobatto)
    top = 2 * n - 1 if pts == nat.GAUSS else 2 * n - 3
    for m in range(top + 1):
        exact = 0.0 if m % 2 else 2.0 / (m + 1)
        assert abs(np.dot(w, t["xi"] ** m) - exact) <= 1e-13


@pytest.mark.parametrize("pts", [nat.GAUSS, nat.LOBATTO])
def test_quadrature_weights_integrate_a_constant_over_the_domain(pts):
    cfg = nat.Config(eqn=nat.EULER, nx=5, ny=3, p=3, x0=-1.0, x1=4.0, y0=0.0, y1=2.0, pts=pts)
    W = adjoint.quadrature_weights(types.SimpleNamespace(cfg=cfg)).cpu().numpy()
    assert W.shape == (4, 15, 16)
    assert np.allclose(W.sum(axis=(1, 2)), 5.0 * 2.0, rtol=1e-13)
