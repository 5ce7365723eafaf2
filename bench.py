#!/usr/bin/env python
"""CPR benchmark: DOF-stage updates/s of the SSP-RK3 CPR solver on GB300.

Workload (one bench "step" = one whole solve): the 2D Euler isentropic vortex
(gamma 1.4, strength 5, centred at (5, 5), mean flow (1, 1)) on the periodic
box [0,10]^2 with 128 x 128 elements, CPR p = 3 (16 Gauss points per element,
4 conserved variables), Rusanov flux, g_DG correction, SSP-RK3 with device-side
CFL steps (CFL 0.08) to t = 10.  The headline value is the FP32 path; the FP64
path runs the same solve once and both report their L2 error of the density
averages against the exact solution (which at t = 10 equals the initial field).

    value = 128 * 128 * 16 * 3 * (RK3 steps) * K / (sum of the K solve times)

summed over ranks (each rank solves its own replica; no data-path collective).
L2 is flushed (a 256 MiB write) before every timed solve, outside its events.
The roofline object covers the dominant kernel (the fused residual + RK stage
kernel): algorithmic bytes per launch (8 state arrays per RK3 step: 8/3 * 4
variables * 4 B = 42.7 B per point and stage) over its mean launch duration;
the FP32 compensated increment form actually moves 10 arrays per step (53.3 B),
reported as moved_gbs.  A second roofline block repeats this on a 1024 x 1024
vortex whose state (268 MB per array) is larger than L2.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "CPR DOF-stage updates/s (FP32 vs FP64, equal L2 error) and % HBM roofline"
UNIT = "DOF-stage/s"
NX, P, L, EPS, T_END, CFL = 128, 3, 10.0, 5.0, 10.0, 0.08
HBM_NX, HBM_STEPS = 1024, 20
# Algorithmic bytes of one DOF-stage (one solution point, all 4 variables):
# the method reads the stage state and writes the next one, and stages 2-3
# also read q^n -- 8 state arrays per RK3 step, 8/3 * 4 variables * 4 B =
# 42.7 B in FP32.  The FP32 path moves more: its compensated increment form
# (stage 1 reads q, writes B1; stage 2 reads q, B1, writes B2; stage 3 reads
# q, B2 and the low part, writes the new high and low parts) moves 10 arrays
# per step (53.3 B per DOF-stage); both are reported.
ALGO_ARRAYS_PER_STEP = 8
MOVED_ARRAYS_PER_STEP = 10
# DRAM bytes (read + write) per stage launch, mean over the three RK stages,
# from ncu captures of the stage kernel as it stands (profiles/): the
# 128^2 workload replayed cold (writes stay in L2) and the 1024^2 case.
NCU_TRAFFIC_128 = 8.429e6
NCU_TRAFFIC_1024 = 8.573e8
FALLBACK_HBM_GBS = 6800.0
# FP64 floating-point operations per DOF-stage of the 128^2 p = 3 Euler stage
# kernel (2 per DFMA, 1 per DMUL / DADD, counted by ncu over the three RK
# stages; IEEE division and square root are DFMA sequences), and the FP64
# peak derived from GB300's units: 152 SMs x 2 FP64 FMA per SM per clock x 2
# flops x 2.07 GHz = 1.26 TFLOP/s (the nominal 1.25).
FP64_FLOPS_PER_DOF_STAGE = 297.4
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12


def f64_roofline(rate):
    if FP64_FLOPS_PER_DOF_STAGE is None:
        return {"bound": "alu", "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s", "achieved": None, "frac": None}
    a = rate * FP64_FLOPS_PER_DOF_STAGE / 1e12
    return {"bound": "alu", "achieved": a, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
            "frac": a / FP64_PEAK_TFLOPS, "flops_per_dof_stage": FP64_FLOPS_PER_DOF_STAGE}


def parse():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["cpr", "reference"], default="cpr")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--workload", choices=["vortex128", "vortex1024", "batch", "fv1536", "limited", "radial", "f64"],
                    default="vortex128", help="vortex1024 / batch / fv1536 / limited / radial / f64: "
                    "only that block (short runs for profiling)")
    ap.add_argument("--no-tune", action="store_true",
                    help="--workload batch: the untuned launch (for profilers, whose serialised replays "
                    "distort the autotuner's timings)")
    ap.add_argument("--quick", action="store_true",
                    help="FP32 timed solves only (no FP64 solve, e2e, HBM case or CPU baseline)")
    return ap.parse_args()


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


def exact_rho_averages(nx):
    """Density averages of the exact solution at t = 10 (= the initial vortex):
    10 x 10 Gauss-Legendre rule on every element."""
    from paper_1709_01619_gb300 import inputs
    g, w = np.polynomial.legendre.leggauss(10)
    h = L / nx
    ii, jj = np.meshgrid(np.arange(nx), np.arange(nx))  # [j, i]
    xs = (ii.ravel()[:, None] + 0.5 * (g[None, :] + 1.0)) * h          # [e, a]
    ys = (jj.ravel()[:, None] + 0.5 * (g[None, :] + 1.0)) * h          # [e, b]
    X = np.repeat(xs[:, None, :], 10, axis=1).reshape(nx * nx, 100)
    Y = np.repeat(ys[:, :, None], 10, axis=2).reshape(nx * nx, 100)
    W = (0.25 * w[:, None] * w[None, :]).reshape(100)                  # [b, a]
    rho = inputs.vortex(X, Y, eps=EPS)[0]
    return rho @ W


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.proc = None
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-i", str(index)],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for name, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "samples": len(sm),
                "reasons": sorted(reasons)}


def dist_setup():
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if torch.cuda.is_available():
        torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def _reduce_over_ranks(x, world, op):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    # NCCL reduces device tensors; gloo (the CPU process groups) host ones
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=op)
    return float(t.item())


def max_over_ranks(x, world):
    import torch.distributed as dist
    return _reduce_over_ranks(x, world, dist.ReduceOp.MAX)


def sum_over_ranks(x, world):
    import torch.distributed as dist
    return _reduce_over_ranks(x, world, dist.ReduceOp.SUM)


# ---------------------------------------------------------------------------
# oracle on the host cores (CPU baseline and the reference arm)
# ---------------------------------------------------------------------------
def oracle_sample(target_s=12.0):
    """Time the FP64 oracle on the 128^2 p=3 vortex for a bounded number of
    SSP-RK3 steps (about target_s seconds).  Returns (DOF-stage/s, steps, s,
    threads)."""
    import oracle
    from paper_1709_01619_gb300 import inputs
    o = oracle.Config(eqn=oracle.EULER, nx=NX, ny=NX, p=P, x1=L, y1=L, cfl=CFL)
    x, y = oracle.point_coords(o)
    q = inputs.vortex(x, y, eps=EPS)
    t0 = time.perf_counter()
    q, _, _ = oracle.run(o, q, 1)
    t1 = time.perf_counter() - t0
    steps = int(max(1, min(400, target_s / max(t1, 1e-6))))
    t0 = time.perf_counter()
    oracle.run(o, q, steps)
    dt = time.perf_counter() - t0
    dof = NX * NX * (P + 1) ** 2
    return dof * 3 * steps / dt, steps, dt, oracle.threads()


def run_reference(args, world, rank):
    if rank != 0:
        return
    per_step_target = max(2.0, 150.0 / max(1, args.steps + args.warmup))
    for _ in range(args.warmup):
        oracle_sample(per_step_target)
    vals, secs, nsteps = [], 0.0, 0
    threads = 1
    for _ in range(args.steps):
        v, s, dt, threads = oracle_sample(per_step_target)
        vals.append(v)
        secs += dt
        nsteps += s
    dof = NX * NX * (P + 1) ** 2
    value = dof * 3 * nsteps / secs
    sample = (f"{nsteps} SSP-RK3 steps of the 128x128 p=3 vortex in FP64 over {args.steps} samples "
              f"(the full solve to t=10 is about 5400 steps)")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * secs / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": "euler_vortex_128x128_p3_t10", "nx": NX, "ny": NX, "p": P,
                   "t_end": T_END, "cfl": CFL, "precision": "fp64", "l2_flush": "n/a (host)"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# CUDA path
# ---------------------------------------------------------------------------
def hbm_case(make, peak, steps=HBM_STEPS):
    """1024^2 p=3 FP32 vortex (268 MB per state array, above L2): the stage
    kernels of `steps` RK3 steps timed back to back with CUDA events."""
    import torch
    from paper_1709_01619_gb300 import _native as nat
    cfgH, ctxH, q0H = make(nat.F32, HBM_NX)
    qH = q0H.clone()
    ctxH.step(qH, 3, 1e-4)
    torch.cuda.synchronize()
    eh = (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
    eh[0].record()
    ctxH.step(qH, steps, 1e-4)
    eh[1].record()
    torch.cuda.synchronize()
    msH = eh[0].elapsed_time(eh[1])
    dofH = HBM_NX * HBM_NX * (P + 1) ** 2
    launchH = msH / (3 * steps)
    achievedH = dofH * 16 * ALGO_ARRAYS_PER_STEP / 3.0 / (launchH * 1e-3) / 1e9
    movedH = achievedH * MOVED_ARRAYS_PER_STEP / ALGO_ARRAYS_PER_STEP
    ctxH.close()
    return {"workload": "euler_vortex_1024x1024_p3_fp32", "bound": "hbm", "achieved": achievedH,
            "peak": peak, "unit": "GB/s", "frac": achievedH / peak, "traffic": NCU_TRAFFIC_1024,
            "moved_gbs": movedH, "moved_frac": movedH / peak, "launch_ms": launchH,
            "dof_stage_per_s": dofH * 3 * steps / (msH * 1e-3), "rk3_steps": steps}


def batch_case(peak, steps=100, warmup=3, tune=True):
    """64 isentropic-vortex instances (N ~ U{32..256}, p ~ U{2,3,4}, strength
    ~ U[1,5], numpy seed 0) on [0,10]^2 in FP32, advanced together by the
    batched solver with per-instance CFL steps after autotuning (tune=False:
    the untuned launch, the grouped form with one CTA per tile of the 8x8
    family, for profilers, whose serialised replays would distort the
    autotuner's timings)."""
    import torch
    from paper_1709_01619_gb300 import _native as nat
    from paper_1709_01619_gb300 import inputs
    specs = inputs.batch_instances(64, seed=0)
    cfgs = [nat.Config(eqn=nat.EULER, nx=s["N"], ny=s["N"], p=s["p"], x1=L, y1=L, dtype=nat.F32,
                       cfl={2: 0.1, 3: 0.08, 4: 0.06}[s["p"]]) for s in specs]
    qs = []
    for c, s in zip(cfgs, specs):
        with nat.Context(c) as ctx:
            x, y = ctx.point_coords()
        qs.append(torch.tensor(inputs.vortex(x, y, eps=s["eps"]), dtype=torch.float32, device="cuda"))
    dof = sum(c.nx * c.ny * (c.p + 1) ** 2 for c in cfgs)
    with nat.Batch(cfgs) as b:
        choices = b.tune(qs) if tune else []
        b.step(qs, warmup)
        torch.cuda.synchronize()
        ev = (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
        ev[0].record()
        b.step(qs, steps)
        ev[1].record()
        torch.cuda.synchronize()
        ms = ev[0].elapsed_time(ev[1])
    rate = dof * 3 * steps / (ms * 1e-3)
    achieved = rate * 16 * ALGO_ARRAYS_PER_STEP / 3.0 / 1e9
    return {"workload": "batch_64_vortex_N32-256_p2-4_fp32", "instances": len(cfgs), "dof": dof,
            "rk3_steps": steps, "ms": ms, "dof_stage_per_s": rate, "bound": "hbm",
            "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
            "tuned": [{"p": p, "family": f, "grid": g} for p, f, g in choices] if tune else None}


def limited_case(peak, fp64_steps=None):
    """Four-quadrant Riemann problem on [0,1]^2 split at (0.8, 0.8), 512^2
    elements, p = 2, TVB minmod limiter (M = 50, eps = 1e-3) after every RK
    stage, transmissive boundaries, CFL 0.1: the FP32 solve to t = 0.3 timed
    whole (the initial condition limited once, outside the timing); FP64 the
    same solve to t = 0.3 (or fp64_steps CFL steps, for short profiling
    runs), and the FP32-vs-FP64 relative L2 difference of the final states."""
    import torch
    from paper_1709_01619_gb300 import _native as nat
    from paper_1709_01619_gb300 import inputs
    nx, p, t_end = 512, 2, 0.3

    def make(dtype):
        cfg = nat.Config(eqn=nat.EULER, nx=nx, ny=nx, p=p, x1=1.0, y1=1.0, bc_x=nat.TRANSMISSIVE,
                         bc_y=nat.TRANSMISSIVE, limiter=1, tvb_M=50.0, lim_eps=1e-3, cfl=0.1, dtype=dtype)
        ctx = nat.Context(cfg)
        x, y = ctx.point_coords()
        q0 = torch.tensor(inputs.four_quadrant(x, y), dtype=cfg.torch_dtype, device="cuda")
        ctx.limit(q0)
        return ctx, q0

    dof = nx * nx * (p + 1) ** 2
    ctx, q0 = make(nat.F32)
    q = q0.clone()
    ctx.set_time(0.0, 0)
    ctx.step(q, 100000, 0.0, t_end)
    nsteps = ctx.get_time()[1]
    q.copy_(q0)
    ctx.set_time(0.0, 0)
    torch.cuda.synchronize()
    ev = (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
    ev[0].record()
    ctx.step(q, nsteps, 0.0, t_end)
    ev[1].record()
    torch.cuda.synchronize()
    ms = ev[0].elapsed_time(ev[1])
    nrm = ctx.norms(q)
    ctx.close()
    rate = dof * 3 * nsteps / (ms * 1e-3)
    # stage kernel (8/3 state arrays per stage) + limiter (reads the state)
    achieved = rate * 16 * (8.0 / 3.0 + 1.0) / 1e9
    ctx64, q64 = make(nat.F64)
    torch.cuda.synchronize()
    ev[0].record()
    if fp64_steps:
        ctx64.step(q64, fp64_steps)
    else:
        ctx64.step(q64, 100000, 0.0, t_end)
    ev[1].record()
    torch.cuda.synchronize()
    ms64 = ev[0].elapsed_time(ev[1])
    n64 = ctx64.get_time()[1]
    out = {"workload": "euler_four_quadrant_512x512_p2_tvb_limiter_t0.3", "rk3_steps": nsteps,
           "ms_fp32": ms, "dof_stage_per_s_fp32": rate, "bound": "hbm", "achieved": achieved, "peak": peak,
           "unit": "GB/s", "frac": achieved / peak,
           "bytes_per_dof_stage": 16 * (8.0 / 3.0 + 1.0),
           "dof_stage_per_s_fp64": dof * 3 * n64 / (ms64 * 1e-3), "fp64_steps_timed": n64,
           "n_marked_final": nrm["n_marked"], "n_nonphys_final": nrm["n_nonphys"]}
    if not fp64_steps:
        a, b = q.double(), q64
        out["ms_fp64"] = ms64
        out["f32_vs_f64_rel_l2"] = float(torch.linalg.norm(a - b) / torch.linalg.norm(b))
        out["f32_vs_f64_rel_l2_rho"] = float(torch.linalg.norm(a[0] - b[0]) / torch.linalg.norm(b[0]))
    ctx64.close()
    return out


def fv_case(peak, fp64_steps=200):
    """The FV run of the equal-DOF comparison: the same four-quadrant problem
    on 1536^2 elements (2,359,296 DOF, as the 512^2 p = 2 CPR run), FV with
    second-order MUSCL and minmod slopes, transmissive, CFL 0.4 (the paper's
    FV CFL), FP32 to t = 0.3 timed whole; FP64 timed over fixed CFL steps."""
    import torch
    from paper_1709_01619_gb300 import _native as nat
    from paper_1709_01619_gb300 import inputs
    n, t_end = 1536, 0.3

    def make(dtype):
        cfg = nat.Config(eqn=nat.EULER, nx=n, ny=n, p=0, x1=1.0, y1=1.0, bc_x=nat.TRANSMISSIVE,
                         bc_y=nat.TRANSMISSIVE, cfl=0.4, dtype=dtype, scheme=nat.SCHEME_FV_MUSCL)
        ctx = nat.Context(cfg)
        x, y = ctx.point_coords()
        return ctx, torch.tensor(inputs.four_quadrant(x, y), dtype=cfg.torch_dtype, device="cuda")

    ctx, q0 = make(nat.F32)
    q = q0.clone()
    ctx.set_time(0.0, 0)
    ctx.step(q, 100000, 0.0, t_end)
    nsteps = ctx.get_time()[1]
    q.copy_(q0)
    ctx.set_time(0.0, 0)
    torch.cuda.synchronize()
    ev = (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
    ev[0].record()
    ctx.step(q, nsteps, 0.0, t_end)
    ev[1].record()
    torch.cuda.synchronize()
    ms = ev[0].elapsed_time(ev[1])
    nrm = ctx.norms(q)
    ctx.close()
    dof = n * n
    rate = dof * 3 * nsteps / (ms * 1e-3)
    achieved = rate * 16 * ALGO_ARRAYS_PER_STEP / 3.0 / 1e9
    ctx64, q64 = make(nat.F64)
    ctx64.step(q64, 5)
    torch.cuda.synchronize()
    ev[0].record()
    ctx64.step(q64, fp64_steps)
    ev[1].record()
    torch.cuda.synchronize()
    ms64 = ev[0].elapsed_time(ev[1])
    ctx64.close()
    cfg3 = nat.Config(eqn=nat.EULER, nx=n, ny=n, p=0, x1=1.0, y1=1.0, bc_x=nat.TRANSMISSIVE,
                      bc_y=nat.TRANSMISSIVE, cfl=0.4, dtype=nat.F32, scheme=nat.SCHEME_FV_MUSCL3)
    x, y = cfg_coords(cfg3)
    ms3, n3, nrm3 = timed_solve(cfg3, inputs.four_quadrant(x, y), t_end)
    return {"workload": "euler_four_quadrant_fv_muscl_1536x1536_t0.3", "dof": dof, "rk3_steps": nsteps,
            "muscl3": {"ms_fp32": ms3, "rk3_steps": n3, "dof_stage_per_s_fp32": dof * 3 * n3 / (ms3 * 1e-3),
                       "n_nonphys_final": nrm3["n_nonphys"]},
            "ms_fp32": ms, "dof_stage_per_s_fp32": rate, "bound": "hbm", "achieved": achieved, "peak": peak,
            "unit": "GB/s", "frac": achieved / peak,
            "note": "state 37.7 MB per array: largely L2-resident",
            "dof_stage_per_s_fp64": dof * 3 * fp64_steps / (ms64 * 1e-3), "fp64_steps_timed": fp64_steps,
            "n_nonphys_final": nrm["n_nonphys"]}


def timed_solve(cfg, q0_np, t_end, limit_first=False):
    """One FP32/FP64 solve to t_end timed whole with CUDA events on the
    context's stream (the step count is found by an untimed solve first).
    Returns (ms, rk3 steps, norms of the result)."""
    import torch
    from paper_1709_01619_gb300 import _native as nat
    with nat.Context(cfg) as ctx:
        q0 = torch.tensor(q0_np, dtype=cfg.torch_dtype, device="cuda")
        if limit_first:
            ctx.limit(q0)
        q = q0.clone()
        ctx.set_time(0.0, 0)
        ctx.step(q, 1000000, 0.0, t_end)
        nsteps = ctx.get_time()[1]
        q.copy_(q0)
        ctx.set_time(0.0, 0)
        torch.cuda.synchronize()
        ev = (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
        ev[0].record()
        ctx.step(q, nsteps, 0.0, t_end)
        ev[1].record()
        torch.cuda.synchronize()
        return ev[0].elapsed_time(ev[1]), nsteps, ctx.norms(q)


def radial_case():
    """The paper's radially expanding shock tube (Sec. 4.2) at the size of
    its P2 timing comparison, 1,440,000 DOF: (rho, p) = (1, 1) inside r < 0.4,
    (0.125, 0.1) outside on [-1, 1]^2, transmissive, FP32 to t = 0.25.  CPR
    400^2 p = 2 with the TVB limiter (M = 50, eps = 1e-3) at CFL 0.1 against
    FV 1200^2 with second- and third-order MUSCL at CFL 0.4: time per RK3
    step and to t = 0.25."""
    from paper_1709_01619_gb300 import _native as nat
    from paper_1709_01619_gb300 import inputs
    t_end = 0.25
    out = {"workload": "euler_radial_shock_tube_1440k_dof_t0.25"}
    common = dict(eqn=nat.EULER, x0=-1.0, x1=1.0, y0=-1.0, y1=1.0, bc_x=nat.TRANSMISSIVE,
                  bc_y=nat.TRANSMISSIVE, dtype=nat.F32)
    cfg = nat.Config(nx=400, ny=400, p=2, limiter=1, tvb_M=50.0, lim_eps=1e-3, cfl=0.1, **common)
    x, y = cfg_coords(cfg)
    ms, n, nrm = timed_solve(cfg, inputs.radial_shock(x, y), t_end, limit_first=True)
    out["cpr_400_p2"] = {"ms": ms, "rk3_steps": n, "ms_per_step": ms / n,
                         "dof_stage_per_s": 400 * 400 * 9 * 3 * n / (ms * 1e-3),
                         "n_marked_final": nrm["n_marked"], "n_nonphys_final": nrm["n_nonphys"]}
    for key, scheme in (("fv_muscl2_1200", nat.SCHEME_FV_MUSCL), ("fv_muscl3_1200", nat.SCHEME_FV_MUSCL3)):
        cfg = nat.Config(nx=1200, ny=1200, p=0, cfl=0.4, scheme=scheme, **common)
        x, y = cfg_coords(cfg)
        ms, n, nrm = timed_solve(cfg, inputs.radial_shock(x, y), t_end)
        out[key] = {"ms": ms, "rk3_steps": n, "ms_per_step": ms / n,
                    "dof_stage_per_s": 1200 * 1200 * 3 * n / (ms * 1e-3), "n_nonphys_final": nrm["n_nonphys"]}
    c, f = out["cpr_400_p2"], out["fv_muscl2_1200"]
    out["cpr_over_fv2_per_step"] = c["ms_per_step"] / f["ms_per_step"]
    out["cpr_over_fv2_time_to_solution"] = c["ms"] / f["ms"]
    return out


def cfg_coords(cfg):
    from paper_1709_01619_gb300 import _native as nat
    with nat.Context(cfg) as ctx:
        return ctx.point_coords()


def paper_setting_case():
    """The CPR variant the paper runs (Gauss-Lobatto solution points, the
    chain-rule flux divergence, Sec. 2.2) on the same 128^2 p = 3 vortex to
    t = 10 in FP32: throughput and the density-average error, next to the
    headline setting (Gauss points, LP divergence)."""
    import torch
    from paper_1709_01619_gb300 import _native as nat
    from paper_1709_01619_gb300 import inputs
    cfg = nat.Config(eqn=nat.EULER, nx=NX, ny=NX, p=P, x1=L, y1=L, cfl=CFL, dtype=nat.F32,
                     pts=nat.LOBATTO, div=nat.DIV_CHAIN)
    with nat.Context(cfg) as ctx:
        x, y = ctx.point_coords()
        q0 = torch.tensor(inputs.vortex(x, y, eps=EPS), dtype=torch.float32, device="cuda")
        q = q0.clone()
        ctx.set_time(0.0, 0)
        ctx.step(q, 20000, 0.0, T_END)
        nsteps = ctx.get_time()[1]
        q.copy_(q0)
        ctx.set_time(0.0, 0)
        torch.cuda.synchronize()
        ev = (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
        ev[0].record()
        ctx.step(q, nsteps, 0.0, T_END)
        ev[1].record()
        torch.cuda.synchronize()
        ms = ev[0].elapsed_time(ev[1])
        avg = ctx.averages(q)[0].double().cpu().numpy()
    # exact averages of the Lobatto run come from the same 10 x 10 rule
    err = float(np.sqrt(np.mean((avg - exact_rho_averages(NX)) ** 2)))
    dof = NX * NX * (P + 1) ** 2
    return {"workload": "euler_vortex_128x128_p3_t10_lobatto_chainrule_fp32", "rk3_steps": nsteps, "ms": ms,
            "dof_stage_per_s": dof * 3 * nsteps / (ms * 1e-3), "l2_rho_avg_error": err}


def adjoint_case():
    """Gradient of J = 1/2 sum W (q_N - q_t)^2 with respect to the initial
    state: Euler vortex (strength 5) on [0,10]^2, 256^2, p = 3, FP32, 400
    SSP-RK3 steps of dt = 7e-4 (t = 0.28, CFL 0.07), checkpoints every 20
    steps, q_t the forward
    solution from strength 4.5.  Forward (with checkpoints) and backward
    (recompute + transposed steps) timed with CUDA events."""
    import torch
    from paper_1709_01619_gb300 import _native as nat
    from paper_1709_01619_gb300 import adjoint, inputs
    n, nsteps, dt, every = 256, 400, 7e-4, 20
    cfg = nat.Config(eqn=nat.EULER, nx=n, ny=n, p=3, x1=L, y1=L, dtype=nat.F32)
    with nat.Context(cfg) as ctx:
        x, y = ctx.point_coords()
        q0 = torch.tensor(inputs.vortex(x, y, eps=EPS), dtype=torch.float32, device="cuda")
        qt = torch.tensor(inputs.vortex(x, y, eps=4.5), dtype=torch.float32, device="cuda")
        ctx.step(qt, nsteps, dt)
        W = adjoint.quadrature_weights(ctx)

        def grad(ev=None):
            q = q0.clone().requires_grad_(True)
            if ev:
                ev[0].record()
            qN = adjoint.rollout(q, ctx, nsteps, dt, every)
            J = 0.5 * (W * (qN - qt) ** 2).sum()
            if ev:
                ev[1].record()
            J.backward()
            if ev:
                ev[2].record()
            return q.grad

        grad()
        torch.cuda.synchronize()
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        g = grad(ev)
        torch.cuda.synchronize()
        fwd, bwd = ev[0].elapsed_time(ev[1]), ev[1].elapsed_time(ev[2])
        finite = bool(torch.isfinite(g).all())
    dof = n * n * 16
    return {"workload": "euler_vortex_256x256_p3_fp32_adjoint_400steps_ckpt20", "forward_ms": fwd,
            "backward_ms": bwd, "gradient_ms": fwd + bwd, "backward_over_forward": bwd / fwd,
            "forward_dof_stage_per_s": dof * 3 * nsteps / (fwd * 1e-3), "gradient_finite": finite}


def run_hbm_only(args):
    import torch
    from paper_1709_01619_gb300 import _native as nat
    from paper_1709_01619_gb300 import inputs
    peak, _ = peaks()

    def make(dtype, nx):
        cfg = nat.Config(eqn=nat.EULER, nx=nx, ny=nx, p=P, x1=L, y1=L, cfl=CFL, dtype=dtype)
        ctx = nat.Context(cfg)
        x, y = ctx.point_coords()
        q0 = torch.tensor(inputs.vortex(x, y, eps=EPS), dtype=cfg.torch_dtype, device="cuda")
        return cfg, ctx, q0

    print(json.dumps(hbm_case(make, peak, max(1, args.steps))), flush=True)


def run_f64_only(args):
    """FP64 path on the 128^2 p = 3 vortex: `steps` CFL RK3 steps timed after
    three untimed ones (a short run for profiling the FP64 stage kernel)."""
    import torch
    from paper_1709_01619_gb300 import _native as nat
    from paper_1709_01619_gb300 import inputs
    cfg = nat.Config(eqn=nat.EULER, nx=NX, ny=NX, p=P, x1=L, y1=L, cfl=CFL, dtype=nat.F64)
    with nat.Context(cfg) as ctx:
        x, y = ctx.point_coords()
        q = torch.tensor(inputs.vortex(x, y, eps=EPS), dtype=torch.float64, device="cuda")
        ctx.step(q, 3)
        torch.cuda.synchronize()
        ev = (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
        ev[0].record()
        ctx.step(q, args.steps)
        ev[1].record()
        torch.cuda.synchronize()
        ms = ev[0].elapsed_time(ev[1])
    dof = NX * NX * (P + 1) ** 2
    rate = dof * 3 * args.steps / (ms * 1e-3)
    print(json.dumps({"workload": "euler_vortex_128x128_p3_fp64", "rk3_steps": args.steps, "ms": ms,
                      "dof_stage_per_s": rate, **f64_roofline(rate)}), flush=True)


def run_cpr(args, world, rank, local):
    import torch
    from paper_1709_01619_gb300 import _native as nat
    from paper_1709_01619_gb300 import inputs

    dof = NX * NX * (P + 1) ** 2
    peak, peak_kind = peaks()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")

    def make(dtype, nx=NX):
        cfg = nat.Config(eqn=nat.EULER, nx=nx, ny=nx, p=P, x1=L, y1=L, cfl=CFL, dtype=dtype)
        ctx = nat.Context(cfg)
        x, y = ctx.point_coords()
        q0 = torch.tensor(inputs.vortex(x, y, eps=EPS), dtype=cfg.torch_dtype, device="cuda")
        return cfg, ctx, q0

    def solve(ctx, q, q0, nsteps, ev=None):
        flush.zero_()
        q.copy_(q0)
        ctx.set_time(0.0, 0)
        if ev:
            ev[0].record()
        ctx.step(q, nsteps, 0.0, T_END)
        if ev:
            ev[1].record()

    # ---- FP32 (headline) ----------------------------------------------------
    cfg32, ctx32, q0_32 = make(nat.F32)
    q32 = torch.empty_like(q0_32)
    solve(ctx32, q32, q0_32, 20000)
    nsteps = ctx32.get_time()[1]
    for _ in range(max(0, args.warmup - 1)):
        solve(ctx32, q32, q0_32, nsteps)
    torch.cuda.synchronize()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(args.steps)]
    clocks = ClockSampler(local)
    barrier(world)
    torch.cuda.synchronize()
    for k in range(args.steps):
        solve(ctx32, q32, q0_32, nsteps, evs[k])
    torch.cuda.synchronize()
    barrier(world)
    clk = clocks.stop()
    ms = sum(a.elapsed_time(b) for a, b in evs)
    t_fin, steps_fin = ctx32.get_time()
    ms_max = max_over_ranks(ms, world)
    updates = dof * 3 * nsteps * args.steps
    value = sum_over_ranks(updates, world) / (ms_max * 1e-3)
    avg32 = ctx32.averages(q32)[0].double().cpu().numpy()

    # dominant kernel: fused residual + stage, 3 launches per RK3 step
    launch_ms = ms / (args.steps * 3 * nsteps)
    bytes_per_launch = dof * 4 * 4 * ALGO_ARRAYS_PER_STEP / 3.0
    achieved = bytes_per_launch / (launch_ms * 1e-3) / 1e9

    if args.quick:
        if rank == 0:
            print(json.dumps({"workload": "euler_vortex_128x128_p3_t10", "value": value, "unit": UNIT,
                              "ms_per_step": ms_max / args.steps, "rk3_steps": nsteps,
                              "launch_ms": launch_ms}), flush=True)
        return

    # ---- e2e through the host-buffer entry point ------------------------------
    qh_in = q0_32.cpu().pin_memory()
    qh_out = torch.empty_like(qh_in).pin_memory()
    ctx32.set_time(0.0, 0)
    ctx32.step_host(qh_in, qh_out, nsteps, 0.0, T_END)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        ctx32.set_time(0.0, 0)
        ctx32.step_host(qh_in, qh_out, nsteps, 0.0, T_END)
    e2e_s = max_over_ranks(time.perf_counter() - t0, world)
    e2e = sum_over_ranks(updates, world) / e2e_s
    state_bytes = qh_in.numel() * 4

    # ---- FP64 path, same solve ----------------------------------------------
    cfg64, ctx64, q0_64 = make(nat.F64)
    q64 = torch.empty_like(q0_64)
    solve(ctx64, q64, q0_64, nsteps + 100)
    n64 = ctx64.get_time()[1]
    ev64 = (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
    solve(ctx64, q64, q0_64, n64, ev64)
    torch.cuda.synchronize()
    ms64 = ev64[0].elapsed_time(ev64[1])
    avg64 = ctx64.averages(q64)[0].cpu().numpy()
    exact = exact_rho_averages(NX)
    err32 = float(np.sqrt(np.mean((avg32 - exact) ** 2)))
    err64 = float(np.sqrt(np.mean((avg64 - exact) ** 2)))
    diff = float(np.linalg.norm(q32.double().cpu().numpy() - q64.cpu().numpy()) /
                 np.linalg.norm(q64.cpu().numpy()))
    value64 = dof * 3 * n64 / (ms64 * 1e-3)
    del ctx64

    hbm = hbm_case(make, peak)
    batch = batch_case(peak)
    limited = limited_case(peak)
    fv = fv_case(peak)
    fv["cpr_512_p2_over_fv_time_to_solution"] = limited["ms_fp32"] / fv["ms_fp32"]
    radial = radial_case()
    adj = adjoint_case()
    paper = paper_setting_case()
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        v, s, secs, thr = oracle_sample(12.0)
        cpu = {"value": v, "unit": UNIT, "cores": thr, "kind": "oracle",
               "sample": f"{s} FP64 SSP-RK3 steps of the same 128x128 p=3 vortex ({secs:.1f} s)"}

    if rank != 0:
        return
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "euler_vortex_128x128_p3_t10", "nx": NX, "ny": NX, "p": P,
                   "points": "gauss", "flux": "rusanov", "t_end": T_END, "cfl": CFL,
                   "rk3_steps_per_solve": nsteps, "t_reached": t_fin,
                   "l2_flush": "256 MiB write before every timed solve",
                   "replicas": world},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": NCU_TRAFFIC_128, "peak_source": peak_kind,
                     "kernel": "cpr_stage_kernel<float,3,Euler,LP,Rusanov> (two-CTA-per-SM instantiation)",
                     "bytes_per_launch": bytes_per_launch,
                     "note": "state (4.2 MB) is L2-resident at this size; traffic from a cold ncu replay"},
        "roofline_hbm_case": hbm,
        "batch": batch,
        "limited": limited,
        "fv_equal_dof": fv,
        "radial_shock_tube": radial,
        "adjoint": adj,
        "paper_setting": paper,
        "f64": {"value": value64, "unit": UNIT, "ms_per_solve": ms64, "rk3_steps": n64,
                "roofline": f64_roofline(value64)},
        "l2_rho_avg_error": {"f32": err32, "f64": err64},
        "f32_vs_f64_rel_l2": diff,
        "speedup_f32_over_f64": value / world / value64 if value64 > 0 else None,
        "e2e": {"value": e2e, "unit": UNIT, "h2d_bytes_per_step": state_bytes,
                "d2h_bytes_per_step": state_bytes},
        "gpu_launches": args.steps * (3 * nsteps + 3),
        "clocks": clk,
        "cpu_baseline": cpu,
    }
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    world, rank, local = dist_setup()
    if args.impl == "reference":
        run_reference(args, world, rank)
    elif args.workload == "vortex1024":
        run_hbm_only(args)
    elif args.workload == "batch":
        print(json.dumps(batch_case(peaks()[0], steps=max(1, args.steps), warmup=args.warmup,
                                    tune=not args.no_tune)), flush=True)
    elif args.workload == "limited":
        print(json.dumps(limited_case(peaks()[0], fp64_steps=max(1, args.steps))), flush=True)
    elif args.workload == "radial":
        print(json.dumps(radial_case()), flush=True)
    elif args.workload == "f64":
        run_f64_only(args)
    elif args.workload == "fv1536":
        print(json.dumps(fv_case(peaks()[0], fp64_steps=max(1, args.steps))), flush=True)
    else:
        run_cpr(args, world, rank, local)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
