"""FP32 CUDA path against the FP64 oracle on the two workloads whose FP32
runs are otherwise checked only indirectly:

* the four-quadrant Riemann problem (Sec. 4.3 setting: 512 x 512 elements,
  p = 2, TVB minmod limiter with M = 50 and eps = 1e-3 after every RK stage,
  transmissive boundaries), run for a fixed number of SSP-RK3 steps in FP32
  and compared with the FP64 oracle run from the same (FP32-rounded) state;
* the 64-instance batch of isentropic vortices (N ~ U{32..256}, p ~ U{2,3,4},
  strength ~ U[1,5], numpy seed 0), every instance compared with its own
  oracle run after a few per-instance CFL steps, in both batch forms.

Tolerance: the FP32 state tolerance, relative L2 <= 1e-5 over every value.
Limiter marks are integers: compared exactly wherever the oracle's marking
margin (the distance of the decisive edge test from its threshold) exceeds
1e-4, far beyond what the FP32 rounding of a few steps can move it.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1709_01619_gb300 import _native as nat
from paper_1709_01619_gb300 import inputs

pytestmark = pytest.mark.gpu

TOL32 = 1e-5
SURE = 1e-4


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


def quadrant_cfgs(nx, ny):
    kw = dict(eqn=nat.EULER, nx=nx, ny=ny, p=2, x1=1.0, y1=1.0, bc_x=nat.TRANSMISSIVE,
              bc_y=nat.TRANSMISSIVE, limiter=1, tvb_M=50.0, lim_eps=1e-3, cfl=0.1)
    c = nat.Config(dtype=nat.F32, **kw)
    o = oracle.Config(eqn=oracle.EULER, nx=nx, ny=ny, p=2, x1=1.0, y1=1.0, bc_x=oracle.TRANSMISSIVE,
                      bc_y=oracle.TRANSMISSIVE, limiter=1, tvb_M=50.0, lim_eps=1e-3, cfl=0.1)
    return c, o


def oracle_last_step(o, q, dt):
    """One limited SSP-RK3 step (Sec. 4; Eq. 35 after every stage) composed
    from the oracle's residual and limiter, returning the marks and margins
    of the third stage's limiter pass with the new state."""
    q1 = oracle.limit(o, q + dt * oracle.residual(o, q))[0]
    q2 = oracle.limit(o, 0.75 * q + 0.25 * (q1 + dt * oracle.residual(o, q1)))[0]
    q3 = q / 3.0 + (2.0 / 3.0) * (q2 + dt * oracle.residual(o, q2))
    ql, marks, margin, _ = oracle.limit(o, q3)
    return ql, marks, margin


@pytest.mark.parametrize("nx,ny,nsteps", [(100, 90, 20), (512, 512, 10)])
def test_four_quadrant_fp32_limited_steps_vs_oracle(nx, ny, nsteps):
    """FP32 limited run (plain Shu-Osher stages, limiter after each) for a
    fixed step count at the step size of the initial state's CFL rule: the
    whole state within 1e-5 of the FP64 oracle, and the final limiter
    pass's marks equal to the oracle's wherever its margin is decisive."""
    c, o = quadrant_cfgs(nx, ny)
    x, y = oracle.point_coords(o)
    q0 = oracle.limit(o, inputs.four_quadrant(x, y))[0]
    q0 = q0.astype(np.float32).astype(np.float64)
    dt = oracle.dt(o, q0)
    q_pre, _, _ = oracle.run(o, q0, nsteps - 1, dt)
    q_or, marks_or, margin = oracle_last_step(o, q_pre, dt)
    with nat.Context(c) as ctx:
        qd = torch.tensor(q0.reshape(c.shape), dtype=torch.float32, device="cuda")
        ctx.step(qd, nsteps, dt)
        marks = ctx.get_marks()
        n_marked = ctx.norms(qd)["n_marked"]
        q = qd.double().cpu().numpy()
    sure = np.abs(margin) > SURE
    assert sure.mean() > 0.95 and marks_or.sum() > 50
    assert np.array_equal(marks[sure], marks_or[sure])
    assert n_marked == marks.sum()
    assert rel_l2(q, q_or) <= TOL32
    # and element by element where the marks agree: no element far off
    agree = marks == marks_or
    err = np.linalg.norm((q - q_or)[:, agree, :], axis=(0, 2))
    scale = np.linalg.norm(q_or[:, agree, :], axis=(0, 2))
    assert float(np.max(err / scale)) <= 1e-4


def batch_workload():
    specs = inputs.batch_instances(64, seed=0)
    cfgs = [nat.Config(eqn=nat.EULER, nx=s["N"], ny=s["N"], p=s["p"], x1=10.0, y1=10.0, dtype=nat.F32,
                       cfl=inputs.BATCH_CFL[s["p"]]) for s in specs]
    ocfgs = [oracle.Config(eqn=oracle.EULER, nx=c.nx, ny=c.ny, p=c.p, x1=10.0, y1=10.0, cfl=c.cfl)
             for c in cfgs]
    q0s = []
    for o, s in zip(ocfgs, specs):
        x, y = oracle.point_coords(o)
        q0s.append(inputs.vortex(x, y, eps=s["eps"]).astype(np.float32).astype(np.float64))
    return cfgs, ocfgs, q0s


@pytest.fixture(scope="module")
def batch_oracle_runs():
    cfgs, ocfgs, q0s = batch_workload()
    runs = [oracle.run(o, q0, 3) for o, q0 in zip(ocfgs, q0s)]
    return cfgs, q0s, runs


@pytest.mark.parametrize("per_instance", [False, True])
def test_batch_64_instances_fp32_vs_oracle(batch_oracle_runs, per_instance):
    """The whole 64-instance FP32 workload, 3 per-instance CFL steps in one
    batched call (compensated increment form), against 64 FP64 oracle runs:
    every instance within 1e-5, with the oracle's step count and a time
    within FP32 rounding of the oracle's."""
    cfgs, q0s, runs = batch_oracle_runs
    qs = [torch.tensor(q0.reshape(c.shape), dtype=torch.float32, device="cuda") for c, q0 in zip(cfgs, q0s)]
    with nat.Batch(cfgs) as b:
        b.set_form(per_instance)
        b.step(qs, 3)
        times = [b.get_time(i) for i in range(len(cfgs))]
    errs = []
    for i, (q, (q_or, n_or, t_or)) in enumerate(zip(qs, runs)):
        assert times[i][1] == n_or == 3, i
        assert times[i][0] == pytest.approx(t_or, rel=1e-5), i
        errs.append(rel_l2(q.double().cpu().numpy(), q_or))
    assert max(errs) <= TOL32, (int(np.argmax(errs)), max(errs))


def test_batch_64_instances_stay_physical_over_500_steps():
    """The per-order CFL numbers of the batch keep every one of the 64
    instances stable: after 500 per-instance CFL steps in FP32 every state
    is finite with positive density and pressure, every simulated time is
    finite, and the vortices have moved (t > 0.2 for the slowest)."""
    cfgs, _, q0s = batch_workload()
    qs = [torch.tensor(q0.reshape(c.shape), dtype=torch.float32, device="cuda") for c, q0 in zip(cfgs, q0s)]
    with nat.Batch(cfgs) as b:
        b.step(qs, 500)
        times = [b.get_time(i) for i in range(len(cfgs))]
    for i, (q, (t, n)) in enumerate(zip(qs, times)):
        assert n == 500 and np.isfinite(t) and t > 0.2, (i, t, n)
        q = q.double()
        rho = q[0]
        p = 0.4 * (q[3] - 0.5 * (q[1] ** 2 + q[2] ** 2) / rho)
        assert bool(torch.isfinite(q).all()) and float(rho.min()) > 0 and float(p.min()) > 0, i
