"""The radially expanding shock tube of Sec. 4.2 in the oracle: (rho, p) =
(1, 1) inside r < 0.4 and (0.125, 0.1) outside on [-1, 1]^2, at rest,
transmissive boundaries.  No exact solution is available here (the paper
compares with a reference curve from Toro); the pins are the symmetries of
the problem, which a correct scheme keeps on a grid symmetric about the
origin: the swap x <-> y (with the two momenta swapped) and the mirror
x -> -x (with rho u negated), positivity, and, on the periodic square (the
same problem until waves cross the boundary), conservation of every
average sum.  With transmissive boundaries the sums are not constant: each
RK stage couples neighbouring elements, so numerical signals of size 1e-5
reach the boundary long before the physical waves do."""
import numpy as np
import pytest

import oracle
from paper_1709_01619_gb300 import inputs

CASES = [
    ("cpr_p2_limited", dict(p=2, limiter=1, tvb_M=50.0, lim_eps=1e-3, cfl=0.1), 16, 1e-13),
    ("cpr_p3_lobatto_limited", dict(p=3, pts=oracle.LOBATTO, limiter=1, tvb_M=50.0, lim_eps=1e-3, cfl=0.05), 12,
     1e-13),
    ("fv_muscl2", dict(p=0, scheme=oracle.FV_MUSCL, cfl=0.4), 40, 0.0),
    ("fv_muscl3", dict(p=0, scheme=oracle.FV_MUSCL3, cfl=0.4), 40, 0.0),
]


@pytest.mark.parametrize("bc", [oracle.TRANSMISSIVE, oracle.PERIODIC])
@pytest.mark.parametrize("name,kw,n,tol", CASES, ids=[c[0] for c in CASES])
def test_radial_shock_keeps_its_symmetries(name, kw, n, tol, bc):
    c = oracle.Config(eqn=oracle.EULER, nx=n, ny=n, x0=-1.0, x1=1.0, y0=-1.0, y1=1.0,
                      bc_x=bc, bc_y=bc, **kw)
    x, y = oracle.point_coords(c)
    q = inputs.radial_shock(x, y)
    if c.limiter:
        q, _, _, _ = oracle.limit(c, q)
    s0 = q.reshape(4, -1).sum(axis=1) if c.p == 0 else oracle.averages(c, q).sum(axis=1)
    q, nst, t = oracle.run(c, q, 12)
    N = c.p + 1
    g = q.reshape(4, n, n, N, N)                    # [v, j, i, b, a]
    gt = g.transpose(0, 2, 1, 4, 3)                 # x <-> y
    assert np.abs(g[0] - gt[0]).max() <= tol and np.abs(g[3] - gt[3]).max() <= tol
    assert np.abs(g[1] - gt[2]).max() <= tol and np.abs(g[2] - gt[1]).max() <= tol
    gm = g[:, :, ::-1, :, ::-1]                     # x -> -x
    assert np.abs(g[0] - gm[0]).max() <= tol and np.abs(g[1] + gm[1]).max() <= tol
    assert np.abs(g[2] - gm[2]).max() <= tol and np.abs(g[3] - gm[3]).max() <= tol
    s1 = q.reshape(4, -1).sum(axis=1) if c.p == 0 else oracle.averages(c, q).sum(axis=1)
    if bc == oracle.PERIODIC:
        assert np.allclose(s1, s0, rtol=1e-13, atol=1e-12)
    assert oracle.norms(c, q)["n_nonphys"] == 0
    assert nst == 12 and t > 0
