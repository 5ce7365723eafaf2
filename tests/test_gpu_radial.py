"""The radially expanding shock tube of Sec. 4.2 on the GPU: parity with the
FP64 oracle for the limited CPR scheme and both FV schemes on small grids,
and the full-size FP32 run of the paper's P2 comparison (400 x 400
elements, p = 2, 1,440,000 DOF) to t = 0.25 checked by the problem's
symmetry (x <-> y with the momenta swapped), positivity and, on the
periodic square, the conservation of the average sums."""
import numpy as np
import pytest
import torch

import oracle
from paper_1709_01619_gb300 import _native as nat
from paper_1709_01619_gb300 import inputs

pytestmark = pytest.mark.gpu

TOL64 = 1e-12
BOX = dict(eqn=nat.EULER, x0=-1.0, x1=1.0, y0=-1.0, y1=1.0)


def make(dtype=nat.F64, **kw):
    c = nat.Config(dtype=dtype, **BOX, **kw)
    o = oracle.Config(eqn=c.eqn, nx=c.nx, ny=c.ny, p=c.p, x0=c.x0, x1=c.x1, y0=c.y0, y1=c.y1,
                      pts=c.pts, flux=c.flux, gamma=c.gamma, bc_x=c.bc_x, bc_y=c.bc_y, limiter=c.limiter,
                      tvb_M=c.tvb_M, lim_eps=c.lim_eps, cfl=c.cfl, scheme=c.scheme)
    return c, o


def rel(a, b):
    a, b = np.asarray(a, np.float64).ravel(), np.asarray(b, np.float64).ravel()
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def dev(q, c):
    return torch.tensor(np.asarray(q).reshape(c.shape), dtype=c.torch_dtype, device="cuda")


def host(t):
    return t.detach().double().cpu().numpy()


@pytest.mark.parametrize("bc", [nat.TRANSMISSIVE, nat.PERIODIC])
def test_limited_cpr_matches_oracle(bc):
    c, o = make(nx=32, ny=32, p=2, bc_x=bc, bc_y=bc, limiter=1, tvb_M=50.0, lim_eps=1e-3, cfl=0.1)
    x, y = oracle.point_coords(o)
    q0, _, _, _ = oracle.limit(o, inputs.radial_shock(x, y))
    q_or, n_or, t_or = oracle.run(o, q0, 8)
    with nat.Context(c) as ctx:
        qd = dev(q0, c)
        ctx.step(qd, 8)
        t, n = ctx.get_time()
        q = host(qd)
    assert n == n_or == 8 and t == pytest.approx(t_or, rel=1e-14)
    assert rel(q, q_or) <= TOL64


@pytest.mark.parametrize("scheme,oscheme", [(nat.SCHEME_FV_MUSCL, oracle.FV_MUSCL),
                                            (nat.SCHEME_FV_MUSCL3, oracle.FV_MUSCL3)])
def test_fv_matches_oracle_to_t_end(scheme, oscheme):
    c, o = make(nx=72, ny=72, p=0, scheme=scheme, bc_x=nat.TRANSMISSIVE, bc_y=nat.TRANSMISSIVE, cfl=0.4)
    assert o.scheme == oscheme
    x, y = oracle.point_coords(o)
    q0 = inputs.radial_shock(x, y)
    q_or, n_or, t_or = oracle.run(o, q0, 100000, 0.0, 0.05)
    with nat.Context(c) as ctx:
        qd = dev(q0, c)
        ctx.step(qd, n_or + 3, 0.0, 0.05)
        t, n = ctx.get_time()
        q = host(qd)
    assert n == n_or and t == t_or == 0.05
    assert rel(q, q_or) <= TOL64


@pytest.mark.parametrize("bc", [nat.TRANSMISSIVE, nat.PERIODIC])
def test_full_size_fp32_run_keeps_symmetry_and_positivity(bc):
    """400 x 400, p = 2, TVB limiter, CFL 0.1, FP32 to t = 0.25.  The FP32
    kernels evaluate the x- and y-lines with the same operations, so the
    diagonal symmetry is kept to rounding: the bound 1e-5 (relative to the
    state's norm) leaves room for a few limiter decisions taken differently
    at mirrored points."""
    n = 400
    c, _ = make(nat.F32, nx=n, ny=n, p=2, bc_x=bc, bc_y=bc, limiter=1, tvb_M=50.0, lim_eps=1e-3, cfl=0.1)
    with nat.Context(c) as ctx:
        x, y = ctx.point_coords()
        qd = torch.tensor(inputs.radial_shock(x, y), dtype=torch.float32, device="cuda")
        ctx.limit(qd)
        s0 = np.array(ctx.norms(qd)["sum_avg"])
        ctx.step(qd, 100000, 0.0, 0.25)
        t, steps = ctx.get_time()
        nrm = ctx.norms(qd)
        q = host(qd)
    assert t == 0.25 and steps > 100
    assert nrm["n_nonphys"] == 0
    g = q.reshape(4, n, n, 3, 3)
    gt = g.transpose(0, 2, 1, 4, 3)
    scale = np.linalg.norm(g)
    err = np.linalg.norm(np.stack([g[0] - gt[0], g[1] - gt[2], g[2] - gt[1], g[3] - gt[3]]))
    assert err <= 1e-5 * scale
    if bc == nat.PERIODIC:
        s1 = np.array(nrm["sum_avg"])
        assert np.allclose(s1[[0, 3]], s0[[0, 3]], rtol=1e-5)
        assert np.abs(s1[1:3]).max() <= 1e-5 * np.abs(s0[0])
