"""Batched solver (cpr_batch_*) against single-problem contexts and the FP64
oracle: uneven grids and orders p = 1..4 in one batch, fixed and per-instance
CFL steps, odd and even step counts (FP32 increment form), autotuning."""
import numpy as np
import pytest
import torch

import oracle
from paper_1709_01619_gb300 import _native as nat
from paper_1709_01619_gb300 import inputs

pytestmark = pytest.mark.gpu

SHAPES = [(9, 7, 1, 3.0), (13, 11, 2, 5.0), (16, 16, 3, 4.0), (10, 13, 4, 2.0), (24, 8, 3, 1.5)]


def cfgs(dtype):
    out = []
    for i, (nx, ny, p, _) in enumerate(SHAPES):
        h = 0.4 + 0.1 * i  # element size differs between instances
        cfl = {1: 0.2, **inputs.BATCH_CFL}[p]  # stable SSP-RK3 CFL per order
        out.append(nat.Config(eqn=nat.EULER, nx=nx, ny=ny, p=p, x1=nx * h, y1=ny * h, cfl=cfl,
                              dtype=dtype))
    return out


def initial(c, eps):
    with nat.Context(c) as ctx:
        x, y = ctx.point_coords()
    q = inputs.vortex(x, y, eps=eps, xc=0.5 * c.x1, yc=0.5 * c.y1, lx=c.x1, ly=c.y1)
    return torch.tensor(q, dtype=c.torch_dtype, device="cuda")


def rel(a, b):
    a, b = a.double(), b.double()
    return float(torch.linalg.norm(a - b) / torch.linalg.norm(b))


TOL = {nat.F64: 1e-12, nat.F32: 2e-6}


def singles(cs, q0s, nsteps, dt, t_end=0.0):
    res, times = [], []
    for c, q0 in zip(cs, q0s):
        with nat.Context(c) as ctx:
            q = q0.clone()
            ctx.step(q, nsteps, dt, t_end)
            res.append(q)
            times.append(ctx.get_time())
    return res, times


@pytest.mark.parametrize("per_instance", [False, True])
@pytest.mark.parametrize("dtype", [nat.F64, nat.F32])
@pytest.mark.parametrize("nsteps", [1, 2, 5, 21])
def test_batch_matches_single_contexts(dtype, nsteps, per_instance):
    """Grouped form: the same arithmetic as single contexts up to the
    kernels' rounding; per-instance form: the single-problem kernels
    themselves, so FP64 states are equal bit for bit (in FP32 a small single
    context takes the stage kernel's two-CTA-per-SM instantiation, which
    the batch does not use, so only the tolerance holds there)."""
    cs = cfgs(dtype)
    q0s = [initial(c, s[3]) for c, s in zip(cs, SHAPES)]
    ref, _ = singles(cs, q0s, nsteps, 0.004)
    with nat.Batch(cs) as b:
        b.set_form(per_instance)
        qs = [q.clone() for q in q0s]
        b.step(qs, nsteps, 0.004)
        for i, (q, r) in enumerate(zip(qs, ref)):
            assert rel(q, r) <= TOL[dtype], i
            if per_instance and dtype == nat.F64:
                assert torch.equal(q, r), i
            assert b.get_time(i)[1] == nsteps


@pytest.mark.parametrize("per_instance", [False, True])
@pytest.mark.parametrize("dtype", [nat.F64, nat.F32])
def test_batch_cfl_run_matches_single_contexts(dtype, per_instance):
    """19 CFL steps (in the per-instance form: a head graph whose chains
    also take each instance's first step size and clear its low part, and a
    tail graph of 11 steps whose chains copy back a state left in the
    stage buffer): the states of single contexts (FP64 per-instance bit for
    bit) and their step counts and times (equal, or within the rounding
    that the CFL step sizes inherit from the states)."""
    cs = cfgs(dtype)
    q0s = [initial(c, s[3]) for c, s in zip(cs, SHAPES)]
    ref, times = singles(cs, q0s, 19, 0.0)
    with nat.Batch(cs) as b:
        b.set_form(per_instance)
        qs = [q.clone() for q in q0s]
        b.step(qs, 19, 0.0)
        for i, (q, r) in enumerate(zip(qs, ref)):
            assert rel(q, r) <= TOL[dtype], i
            if per_instance and dtype == nat.F64:
                assert torch.equal(q, r), i
            t, n = b.get_time(i)
            assert n == times[i][1] == 19
            # the step sizes follow the states' rounding (FP32, grouped form)
            if per_instance and dtype == nat.F64:
                assert t == times[i][0]
            else:
                assert abs(t - times[i][0]) <= 1e-6 * times[i][0]


def test_per_instance_form_follows_new_state_arrays():
    """The per-instance graphs hold the state pointers: stepping other
    arrays re-captures them."""
    cs = cfgs(nat.F32)
    q0s = [initial(c, s[3]) for c, s in zip(cs, SHAPES)]
    ref, _ = singles(cs, q0s, 3, 0.004)
    with nat.Batch(cs) as b:
        b.set_form(True)
        qa = [q.clone() for q in q0s]
        b.step(qa, 3, 0.004)
        b.set_time(0.0, 0)
        qb = [q.clone() for q in q0s]
        b.step(qb, 3, 0.004)
        for a, c, r in zip(qa, qb, ref):
            assert torch.equal(a, c) and rel(a, r) <= TOL[nat.F32]


def test_batch_matches_oracle_fp64():
    cs = cfgs(nat.F64)[:3]
    with nat.Batch(cs) as b:
        q0s = [initial(c, s[3]) for c, s in zip(cs, SHAPES)]
        qs = [q.clone() for q in q0s]
        b.step(qs, 3, 0.005)
    for c, q0, q in zip(cs, q0s, qs):
        o = oracle.Config(eqn=oracle.EULER, nx=c.nx, ny=c.ny, p=c.p, x1=c.x1, y1=c.y1)
        q_or, _, _ = oracle.run(o, q0.cpu().numpy(), 3, 0.005)
        assert np.linalg.norm(q.cpu().numpy() - q_or) / np.linalg.norm(q_or) <= 1e-12


@pytest.mark.parametrize("per_instance", [False, True])
@pytest.mark.parametrize("dtype", [nat.F64, nat.F32])
def test_batch_cfl_steps_per_instance_to_t_end(dtype, per_instance):
    cs = cfgs(dtype)
    # a smooth periodic solution: rounding differences between the two paths
    # are not amplified by the flow (a vortex cut off by the small periodic
    # boxes develops sharp fronts)
    q0s = []
    for c in cs:
        with nat.Context(c) as ctx:
            x, y = ctx.point_coords()
        q0s.append(torch.tensor(inputs.entropy_wave(x, y, c.x1, c.y1), dtype=c.torch_dtype, device="cuda"))
    t_end = 0.3
    ref, times = singles(cs, q0s, 200, 0.0, t_end)
    with nat.Batch(cs) as b:
        b.set_form(per_instance)
        qs = [q.clone() for q in q0s]
        b.step(qs, 200, 0.0, t_end)
        for i in range(len(cs)):
            t, n = b.get_time(i)
            assert t == t_end and n == times[i][1]
            assert rel(qs[i], ref[i]) <= TOL[dtype]
    assert len(set(n for _, n in times)) > 1  # the instances took different step counts


def test_batch_tune_keeps_states_and_results():
    cs = cfgs(nat.F32)
    q0s = [initial(c, s[3]) for c, s in zip(cs, SHAPES)]
    with nat.Batch(cs) as b:
        qs = [q.clone() for q in q0s]
        choices = b.tune(qs)
        assert {p for p, _, _ in choices} == {1, 2, 3, 4}
        # a tile family and grid per group, or family 2 (per-instance form)
        assert all((f in (0, 1) and g >= 1) or (f == 2 and g == 0) for _, f, g in choices)
        assert len({f == 2 for _, f, _ in choices}) == 1
        for q, q0 in zip(qs, q0s):
            assert torch.equal(q, q0)
        assert b.get_time(0) == (0.0, 0)
        b.step(qs, 4, 0.004)
    ref, _ = singles(cs, q0s, 4, 0.004)
    for q, r in zip(qs, ref):
        assert rel(q, r) <= TOL[nat.F32]


def test_batch_step_host_matches_device_step():
    """cpr_batch_step_host (host buffers, copies inside the call) gives the
    states of cpr_batch_step on device arrays, on two calls in a row."""
    cs = cfgs(nat.F32)
    q0s = [initial(c, s[3]) for c, s in zip(cs, SHAPES)]
    with nat.Batch(cs) as b:
        qd = [q.clone() for q in q0s]
        b.step(qd, 3, 0.004)
        b.step(qd, 2, 0.004)
    with nat.Batch(cs) as b:
        hin = [q.cpu().pin_memory() for q in q0s]
        hout = [torch.empty_like(h).pin_memory() for h in hin]
        b.step_host(hin, hout, 3, 0.004)
        b.step_host(hout, hout, 2, 0.004)
        assert all(b.get_time(i)[1] == 5 for i in range(len(cs)))
    for d, h in zip(qd, hout):
        assert torch.equal(d.cpu(), h)


@pytest.mark.parametrize("dtype", [nat.F32, nat.F64])
@pytest.mark.parametrize("nsteps,dt,t_end", [(21, 0.0, 0.0), (37, 0.0, 0.0), (16, 0.004, 0.0), (40, 0.0, 0.05)])
def test_batch_step_host_overlapped_matches_device_step(dtype, nsteps, dt, t_end):
    """The host entry point in the per-instance form with page-locked
    buffers (copies in the chains of a head and a tail graph, overlapping
    other instances' steps) against the device entry point: the same
    states bit for bit, step counts and times, for CFL and fixed steps, an
    end time that stops instances early, odd and even tails, and two calls
    in a row (the second one reusing the graphs bound to the buffers); then
    pageable buffers, which take the plain path, the same again."""
    cs = cfgs(dtype)
    q0s = [initial(c, s[3]) for c, s in zip(cs, SHAPES)]
    with nat.Batch(cs) as b:
        b.set_form(True)
        qd = [q.clone() for q in q0s]
        b.step(qd, nsteps, dt, t_end)
        td = [b.get_time(i) for i in range(len(cs))]
        b.set_time(0.0, 0)
        b.step(qd, nsteps, dt, t_end)
        td2 = [b.get_time(i) for i in range(len(cs))]
    with nat.Batch(cs) as b:
        b.set_form(True)
        hin = [q.cpu().pin_memory() for q in q0s]
        hout = [torch.empty_like(h).pin_memory() for h in hin]
        b.step_host(hin, hout, nsteps, dt, t_end)
        assert [b.get_time(i) for i in range(len(cs))] == td
        b.set_time(0.0, 0)
        b.step_host(hout, hout, nsteps, dt, t_end)
        assert [b.get_time(i) for i in range(len(cs))] == td2
        for d, h in zip(qd, hout):
            assert torch.equal(d.cpu(), h)
        pin = [q.cpu() for q in q0s]
        pout = [torch.empty_like(h) for h in pin]
        b.set_time(0.0, 0)
        b.step_host(pin, pout, nsteps, dt, t_end)
        b.set_time(0.0, 0)
        b.step_host(pout, pout, nsteps, dt, t_end)
        for d, h in zip(qd, pout):
            assert torch.equal(d.cpu(), h)
