#!/usr/bin/env python
"""CPR benchmark: DOF-stage updates/s of the SSP-RK3 CPR solver on GB300.

Headline workload (one bench "step" = one pass of the whole hot path over
one batch of synthetic input): 64 isentropic-vortex problems of the 2D Euler
equations (gamma 1.4, mean flow (1, 1), centred at (5, 5) on the periodic box
[0,10]^2; per instance N x N elements with N ~ U{32..256}, CPR order
p ~ U{2,3,4}, vortex strength ~ U[1,5], all drawn from numpy seed 0), Gauss
points, Rusanov flux, g_DG correction, advanced together by the batched
solver for 100 SSP-RK3 steps with per-instance device-side CFL steps
(CFL 0.1 / 0.06 / 0.04 for p = 2 / 3 / 4, below the stability bound), FP32 state with the compensated
increment form, FP64 time and reductions.  The autotuner picks the batch
form before the timed region.  Each timed pass starts from the same initial
states (reset outside the timed events); the states (445 MB per array) are
larger than L2.

    value = sum_i N_i^2 (p_i+1)^2 * 3 * 100 * K / (sum of the K pass times)

summed over ranks (each rank advances its own replica of the batch; no
data-path collective).  The roofline object covers the stage kernels, the
dominant kernels of the pass: algorithmic bytes of one batch stage (8 state
arrays per RK3 step: 8/3 * 4 variables * 4 B = 42.7 B per DOF) over the mean
time of one batch stage; the compensated FP32 form moves 10 arrays per step.
`e2e` is the same pass through cpr_batch_step_host with pinned host buffers
(every state copied in and the results copied out inside the timed region).

Beside it (compact keys, full records on stderr): the single-problem stage
kernel on the 1024^2 p = 3 vortex (268 MB per array), the 128^2 p = 3 vortex
to t = 10 in FP32 and FP64 with both density-average errors, the time to a
given error of FP32 and FP64 over a ladder of grids, the limited four-quadrant
run, the FV equal-DOF runs, the radial shock tube, the adjoint, the paper's
point set and divergence, and the oracle on the host cores.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import platform
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
WORKLOAD = "batch_64_euler_vortex_N32-256_p2-4_fp32_100_rk3_steps"
BATCH_N, BATCH_SEED, BATCH_STEPS = 64, 0, 100
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
# from ncu captures of the stage kernel (profiles/): the 128^2 workload
# replayed cold (writes stay in L2) and the 1024^2 case.
NCU_TRAFFIC_128 = 8.429e6
NCU_TRAFFIC_1024 = 8.575e8
FALLBACK_HBM_GBS = 6800.0
# FP64 floating-point operations per DOF-stage of the Euler LP stage at
# p = 3: the method's own count (point fluxes about 25, the two line
# derivatives 4 V n 2 = 128, the correction 4 V 2 = 32 and the face fluxes
# about 60 per face point, 60 * 4n / n^2 = 15; about 200), and the count the
# FP64 stage kernel executes (2 per DFMA, 1 per DMUL / DADD, counted by ncu
# over the three RK stages of the 128^2 p = 3 vortex: 297.4, with index
# arithmetic in FP64 and IEEE division and square root as DFMA sequences).
# The FP64 peak is derived from GB300's units, not measured: 152 SMs x 2 FP64
# FMA per SM per clock x 2 flops x 2.07 GHz = 1.26 TFLOP/s (the nominal 1.25).
FP64_FLOPS_ALGO = 200.0
FP64_FLOPS_EXECUTED = 297.4
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12
# Coarser grids of the equal-error ladder (p = 3 vortex to t = 10, beside 128^2).
LADDER = (24, 32, 48, 64, 96)


def f64_roofline(rate):
    a = rate * FP64_FLOPS_ALGO / 1e12
    return {"bound": "alu", "achieved": a, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
            "frac": a / FP64_PEAK_TFLOPS, "flops_per_dof_stage": FP64_FLOPS_ALGO,
            "executed_flops_per_dof_stage": FP64_FLOPS_EXECUTED,
            "executed_frac": rate * FP64_FLOPS_EXECUTED / 1e12 / FP64_PEAK_TFLOPS,
            "peak_source": "derived from unit counts and clock, not measured"}


def parse():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["cpr", "reference"], default="cpr")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--workload", choices=["headline", "vortex128", "vortex1024", "batch", "fv1536", "limited",
                                           "radial", "f64", "ladder", "adjoint", "vjp"],
                    default="headline", help="anything but headline: only that block (short runs for "
                    "profiling)")
    ap.add_argument("--p", type=int, default=P, help="--workload vortex1024: the order")
    ap.add_argument("--per-instance", action="store_true",
                    help="--workload batch --no-tune: the per-instance chains instead of grouped launches")
    ap.add_argument("--no-tune", action="store_true",
                    help="--workload batch: the untuned launch (for profilers, whose serialised replays "
                    "distort the autotuner's timings)")
    ap.add_argument("--quick", action="store_true", help="the headline only (no side blocks, no CPU baseline)")
    return ap.parse_args()


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


def compact(x, sig=4):
    """Floats rounded to `sig` significant digits, recursively (the printed line)."""
    if isinstance(x, float):
        if x == 0.0 or not math.isfinite(x):
            return x
        return float(f"{x:.{sig}g}")
    if isinstance(x, dict):
        return {k: compact(v, sig) for k, v in x.items()}
    if isinstance(x, (list, tuple)):
        return [compact(v, sig) for v in x]
    return x


def cpu_model():
    """The host CPU's model name (x86 /proc/cpuinfo, else lscpu, else platform)."""
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith("model name"):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    return platform.processor() or platform.machine()


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
# the headline workload: 64 ragged vortex instances
# ---------------------------------------------------------------------------
def batch_specs():
    from paper_1709_01619_gb300 import inputs
    return inputs.batch_instances(BATCH_N, seed=BATCH_SEED)


def batch_dof(specs=None):
    specs = specs or batch_specs()
    return sum(s["N"] * s["N"] * (s["p"] + 1) ** 2 for s in specs)


# ---------------------------------------------------------------------------
# oracle on the host cores (CPU baseline and the reference arm)
# ---------------------------------------------------------------------------
def oracle_batch_states(every=1):
    """Oracle configurations and FP64 initial states of every `every`-th
    instance of the headline batch."""
    import oracle
    from paper_1709_01619_gb300 import inputs
    out = []
    for s in batch_specs()[::every]:
        o = oracle.Config(eqn=oracle.EULER, nx=s["N"], ny=s["N"], p=s["p"], x1=L, y1=L, cfl=inputs.BATCH_CFL[s["p"]])
        x, y = oracle.point_coords(o)
        out.append((o, inputs.vortex(x, y, eps=s["eps"])))
    return out


def oracle_batch_sample(steps=1, every=1, threads=None, states=None):
    """Time the FP64 oracle on `steps` CFL RK3 steps of every `every`-th
    instance of the headline batch (the initial states built outside the
    timing).  threads: OpenMP threads for the sample (None: all).
    Returns (DOF-stage/s, DOF-stages, s, threads used)."""
    import oracle
    states = states if states is not None else oracle_batch_states(every)
    prev = oracle.threads()
    if threads:
        oracle.set_threads(threads)
    try:
        used = oracle.threads()
        work = 0
        t0 = time.perf_counter()
        for o, q in states:
            oracle.run(o, q, steps)
            work += o.ne * o.n * o.n * 3 * steps
        secs = time.perf_counter() - t0
    finally:
        oracle.set_threads(prev)
    return work / secs, work, secs, used


def run_reference(args, world, rank):
    """The reference arm: the FP64 oracle (the plain CPU restatement of the
    method that the tests check the CUDA path against) on the host cores,
    each step one CFL RK3 step of all 64 instances of the headline batch."""
    if rank != 0:
        return
    states = oracle_batch_states()
    for _ in range(args.warmup):
        oracle_batch_sample(1, states=states)
    work, secs, threads = 0, 0.0, 1
    for _ in range(args.steps):
        _, w, s, threads = oracle_batch_sample(1, states=states)
        work += w
        secs += s
    value = work / secs
    sample = (f"1 FP64 SSP-RK3 CFL step of all 64 instances per bench step, {args.steps} steps "
              f"(the GPU arm advances each pass by {BATCH_STEPS} steps)")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * secs / max(1, args.steps),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "instances": BATCH_N, "seed": BATCH_SEED, "dof": batch_dof(),
                   "precision": "fp64", "l2_flush": "n/a (host)"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                         "sample": sample, "cpu": cpu_model()},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(compact(line)), flush=True)


# ---------------------------------------------------------------------------
# CUDA path
# ---------------------------------------------------------------------------
def batch_inputs(specs=None):
    """Configurations and FP32 device initial states of the headline batch."""
    import torch
    from paper_1709_01619_gb300 import _native as nat
    from paper_1709_01619_gb300 import inputs
    specs = specs or batch_specs()
    cfgs = [nat.Config(eqn=nat.EULER, nx=s["N"], ny=s["N"], p=s["p"], x1=L, y1=L, dtype=nat.F32,
                       cfl=inputs.BATCH_CFL[s["p"]]) for s in specs]
    q0s = []
    for c, s in zip(cfgs, specs):
        with nat.Context(c) as ctx:
            x, y = ctx.point_coords()
        q0s.append(torch.tensor(inputs.vortex(x, y, eps=s["eps"]), dtype=torch.float32, device="cuda"))
    return cfgs, q0s


def batch_headline(args, world, local, peak):
    """The headline: K timed passes of the batch (BATCH_STEPS CFL steps each)
    after autotuning and W untimed passes; then the same passes through the
    host-buffer entry point for e2e."""
    import torch
    from paper_1709_01619_gb300 import _native as nat
    cfgs, q0s = batch_inputs()
    dof = batch_dof()
    qs = [q.clone() for q in q0s]
    out = {}
    with nat.Batch(cfgs) as b:
        choices = b.tune(qs)
        per_inst = bool(choices) and choices[0][1] == 2
        ngroups = len(choices)

        def reset():
            for q, q0 in zip(qs, q0s):
                q.copy_(q0)
            b.set_time(0.0, 0)

        for _ in range(args.warmup):
            reset()
            b.step(qs, BATCH_STEPS)
        torch.cuda.synchronize()
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(args.steps)]
        clocks = ClockSampler(local)
        barrier(world)
        torch.cuda.synchronize()
        for k in range(args.steps):
            reset()
            evs[k][0].record()
            b.step(qs, BATCH_STEPS)
            evs[k][1].record()
        torch.cuda.synchronize()
        barrier(world)
        clk = clocks.stop()
        ms = sum(a.elapsed_time(e) for a, e in evs)
        steps_done = [b.get_time(i)[1] for i in range(len(cfgs))]
        t_reached = [b.get_time(i)[0] for i in range(len(cfgs))]
        finite = all(bool(torch.isfinite(q).all()) for q in qs)

        # e2e: the same pass through cpr_batch_step_host, pinned host buffers
        hin = [q.cpu().pin_memory() for q in q0s]
        hout = [torch.empty_like(h).pin_memory() for h in hin]
        b.set_time(0.0, 0)
        b.step_host(hin, hout, BATCH_STEPS)
        clocks_e2e = ClockSampler(local)
        t0 = time.perf_counter()
        for _ in range(args.steps):
            b.set_time(0.0, 0)
            b.step_host(hin, hout, BATCH_STEPS)
        e2e_s = time.perf_counter() - t0
        clk_e2e = clocks_e2e.stop()
        e2e_equal = all(torch.equal(h, q.cpu()) for h, q in zip(hout, qs))
    ms_max = max_over_ranks(ms, world)
    updates = dof * 3 * BATCH_STEPS * args.steps
    value = sum_over_ranks(updates, world) / (ms_max * 1e-3)
    e2e = sum_over_ranks(updates, world) / max_over_ranks(e2e_s, world)
    stage_ms = ms / (args.steps * 3 * BATCH_STEPS)
    bytes_per_stage = dof * 16 * ALGO_ARRAYS_PER_STEP / 3.0
    achieved = bytes_per_stage / (stage_ms * 1e-3) / 1e9
    state_bytes = dof * 16
    kernels_per_step = 3 * (len(cfgs) if per_inst else ngroups)
    out.update(
        value=value, ms=ms, ms_max=ms_max, dof=dof, clocks=clk, clocks_e2e=clk_e2e, finite=finite,
        steps_done=steps_done,
        t_min=min(t_reached), t_max=max(t_reached), e2e=e2e, e2e_equal=e2e_equal, state_bytes=state_bytes,
        tuned=[{"p": p, "family": f, "grid": g} for p, f, g in choices], per_instance=per_inst,
        roofline={"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                  "traffic": None, "unit_of_work": "one batch stage (all 64 instances)",
                  "bytes_per_stage": bytes_per_stage, "stage_ms": stage_ms,
                  "moved_frac": achieved * MOVED_ARRAYS_PER_STEP / ALGO_ARRAYS_PER_STEP / peak,
                  "kernel": "cpr_stage_kernel<float,p,Euler,LP,Rusanov> (p = 2, 3, 4)"},
        # per pass: the stage kernels, the configure kernel, one first-CFL
        # pass per instance and one parity-copy kernel per order group
        gpu_launches=args.steps * (BATCH_STEPS * kernels_per_step + 1 + len(cfgs) + ngroups))
    return out


def hbm_case(make, peak, steps=HBM_STEPS, p=P):
    """1024^2 FP32 vortex of order p (p = 3: 268 MB per state array, above
    L2): the stage kernels of `steps` RK3 steps timed back to back with CUDA
    events."""
    import torch
    from paper_1709_01619_gb300 import _native as nat
    cfgH, ctxH, q0H = make(nat.F32, HBM_NX, p)
    qH = q0H.clone()
    ctxH.step(qH, 3, 1e-4)
    torch.cuda.synchronize()
    eh = (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
    eh[0].record()
    ctxH.step(qH, steps, 1e-4)
    eh[1].record()
    torch.cuda.synchronize()
    msH = eh[0].elapsed_time(eh[1])
    dofH = HBM_NX * HBM_NX * (p + 1) ** 2
    launchH = msH / (3 * steps)
    achievedH = dofH * 16 * ALGO_ARRAYS_PER_STEP / 3.0 / (launchH * 1e-3) / 1e9
    movedH = achievedH * MOVED_ARRAYS_PER_STEP / ALGO_ARRAYS_PER_STEP
    ctxH.close()
    return {"workload": f"euler_vortex_{HBM_NX}x{HBM_NX}_p{p}_fp32", "bound": "hbm", "achieved": achievedH,
            "peak": peak, "unit": "GB/s", "frac": achievedH / peak,
            "traffic": NCU_TRAFFIC_1024 if p == 3 else None,
            "moved_gbs": movedH, "moved_frac": movedH / peak, "launch_ms": launchH,
            "dof_stage_per_s": dofH * 3 * steps / (msH * 1e-3), "rk3_steps": steps}


def make_vortex(dtype, nx=NX, p=P):
    import torch
    from paper_1709_01619_gb300 import _native as nat
    from paper_1709_01619_gb300 import inputs
    cfg = nat.Config(eqn=nat.EULER, nx=nx, ny=nx, p=p, x1=L, y1=L, cfl=CFL, dtype=dtype)
    ctx = nat.Context(cfg)
    x, y = ctx.point_coords()
    q0 = torch.tensor(inputs.vortex(x, y, eps=EPS), dtype=cfg.torch_dtype, device="cuda")
    return cfg, ctx, q0


def vortex_solve(dtype, nx, p=P, repeats=1, flush=None):
    """The vortex on nx^2 elements of order p solved to t = 10 (CFL steps on
    the device): the step count from an untimed solve, then `repeats` timed
    solves from the initial state (L2 flushed before each when given).
    Returns (mean ms, RK3 steps, density-average error, final state)."""
    import torch
    cfg, ctx, q0 = make_vortex(dtype, nx, p)
    with ctx:
        q = q0.clone()
        ctx.set_time(0.0, 0)
        ctx.step(q, 1000000, 0.0, T_END)
        nsteps = ctx.get_time()[1]
        ms = []
        for _ in range(repeats):
            if flush is not None:
                flush.zero_()
            q.copy_(q0)
            ctx.set_time(0.0, 0)
            ev = (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
            ev[0].record()
            ctx.step(q, nsteps, 0.0, T_END)
            ev[1].record()
            torch.cuda.synchronize()
            ms.append(ev[0].elapsed_time(ev[1]))
        avg = ctx.averages(q)[0].double().cpu().numpy()
    err = float(np.sqrt(np.mean((avg - exact_rho_averages(nx)) ** 2)))
    return statistics.mean(ms), nsteps, err, q


def vortex128_case(peak):
    """The 128^2 p = 3 vortex to t = 10 (5348 RK3 steps), FP32 and FP64: time
    to solution, the density-average errors against the exact solution, the
    FP32-vs-FP64 difference, and the stage kernel's roofline (its state is
    L2-resident at this size)."""
    import torch
    from paper_1709_01619_gb300 import _native as nat
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    ms32, n32, err32, q32 = vortex_solve(nat.F32, NX, repeats=3, flush=flush)
    ms64, n64, err64, q64 = vortex_solve(nat.F64, NX, repeats=1, flush=flush)
    diff = float(torch.linalg.norm(q32.double() - q64) / torch.linalg.norm(q64))
    dof = NX * NX * (P + 1) ** 2
    launch_ms = ms32 / (3 * n32)
    achieved = dof * 16 * ALGO_ARRAYS_PER_STEP / 3.0 / (launch_ms * 1e-3) / 1e9
    r64 = dof * 3 * n64 / (ms64 * 1e-3)
    return {"workload": "euler_vortex_128x128_p3_t10", "rk3_steps": n32, "ms_fp32": ms32,
            "dof_stage_per_s_fp32": dof * 3 * n32 / (ms32 * 1e-3), "ms_fp64": ms64,
            "dof_stage_per_s_fp64": r64, "same_grid_f32_over_f64": ms64 / ms32,
            "l2_rho_avg_error": {"f32": err32, "f64": err64}, "f32_vs_f64_rel_l2": diff,
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "frac": achieved / peak,
                         "traffic": NCU_TRAFFIC_128, "launch_ms": launch_ms,
                         "note": "state 4.2 MB: L2-resident, launch-latency bound"},
            "f64_roofline": f64_roofline(r64)}


def loglog(xs, ys, x):
    """Piecewise-linear interpolation of log y over log x (xs decreasing or
    increasing); None outside the range."""
    pts = sorted(zip(xs, ys))
    for (x0, y0), (x1, y1) in zip(pts, pts[1:]):
        if x0 <= x <= x1:
            if x1 == x0:
                return y0
            f = (math.log(x) - math.log(x0)) / (math.log(x1) - math.log(x0))
            return math.exp(math.log(y0) + f * (math.log(y1) - math.log(y0)))
    return None


def time_to_error(rows, target):
    """Least time in which a ladder of runs (dicts with 'ms' and 'err')
    reaches error `target`: the runs that no cheaper run beats in error (the
    time-error frontier), interpolated log-log along it; None when no run
    reaches the target, and the cheapest run's time when it already does."""
    front = []
    for r in sorted(rows, key=lambda r: r["ms"]):
        if not front or r["err"] < front[-1]["err"]:
            front.append(r)
    if front[0]["err"] <= target:
        return front[0]["ms"]
    return loglog([r["err"] for r in front], [r["ms"] for r in front], target)


def equal_error_case(v128):
    """Time to solution at equal error: the 128^2 p = 3 vortex to t = 10 and
    the same problem on coarser grids (LADDER), FP32 and FP64, each with its
    density-average error against the exact solution.  Two readings: (a) the
    FP32 128^2 run against the FP64 time interpolated (log time over log
    error) to its error along the FP64 ladder; (b) at given errors, the least
    time each precision needs along its time-error frontier (FP32 stops
    improving at its rounding floor, about 7e-7, so below that only FP64
    reaches the error)."""
    from paper_1709_01619_gb300 import _native as nat
    rows = {}
    for key, dt in (("f32", nat.F32), ("f64", nat.F64)):
        rows[key] = []
        for n in LADDER:
            ms, steps, err, _ = vortex_solve(dt, n, repeats=2 if n < 96 else 1)
            rows[key].append({"n": n, "ms": ms, "rk3_steps": steps, "err": err})
        # the 128^2 solves of the vortex128 block
        rows[key].append({"n": NX, "ms": v128[f"ms_{key.replace('f', 'fp')}"], "rk3_steps": v128["rk3_steps"],
                          "err": v128["l2_rho_avg_error"][key]})
    out = {"workload": "euler_vortex_p3_t10_grid_ladder", "ladder": rows}
    e32 = rows["f32"][-1]["err"]
    t32 = rows["f32"][-1]["ms"]
    t64 = loglog([r["err"] for r in rows["f64"]], [r["ms"] for r in rows["f64"]], e32)
    out["f32_128_run"] = {"error": e32, "f32_ms": t32, "f64_ms": t64,
                          "speedup_f32_over_f64": (t64 / t32) if t64 else None}
    out["frontier"] = {}
    for target in (e32, 1e-6, 3e-6):
        a = time_to_error(rows["f32"], target)
        c = time_to_error(rows["f64"], target)
        out["frontier"][f"{target:.3g}"] = {"f32_ms": a, "f64_ms": c,
                                            "speedup_f32_over_f64": (c / a) if a and c else None}
    return out


def batch_case(peak, steps=100, warmup=3, tune=True, per_instance=False):
    """64 isentropic-vortex instances (N ~ U{32..256}, p ~ U{2,3,4}, strength
    ~ U[1,5], numpy seed 0) on [0,10]^2 in FP32, advanced together by the
    batched solver with per-instance CFL steps after autotuning (tune=False:
    untuned, the grouped form with one CTA per tile of the 8x8 family, or
    with per_instance the per-instance chains, the form the autotuner picks
    on GB300; for profilers, whose serialised replays would distort the
    autotuner's timings)."""
    import torch
    from paper_1709_01619_gb300 import _native as nat
    from paper_1709_01619_gb300 import inputs
    specs = inputs.batch_instances(64, seed=0)
    cfgs = [nat.Config(eqn=nat.EULER, nx=s["N"], ny=s["N"], p=s["p"], x1=L, y1=L, dtype=nat.F32,
                       cfl=inputs.BATCH_CFL[s["p"]]) for s in specs]
    qs = []
    for c, s in zip(cfgs, specs):
        with nat.Context(c) as ctx:
            x, y = ctx.point_coords()
        qs.append(torch.tensor(inputs.vortex(x, y, eps=s["eps"]), dtype=torch.float32, device="cuda"))
    dof = sum(c.nx * c.ny * (c.p + 1) ** 2 for c in cfgs)
    with nat.Batch(cfgs) as b:
        choices = b.tune(qs) if tune else []
        if not tune and per_instance:
            b.set_form(True)
        b.step(qs, warmup)
        if steps >= 16:
            # runs of 16 steps or more take per-instance head and tail graphs,
            # captured on first use: once outside the timing
            b.step(qs, steps)
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
    same solve to t = 0.3, and the FP32-vs-FP64 relative L2 difference of the
    final states.  fp64_steps: only that many CFL steps in both precisions
    (short runs for profiling)."""
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
    if fp64_steps:
        nsteps = fp64_steps  # a short run of both precisions (profiling)
    else:
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


def vjp_case(peak, reps=10, n=1024):
    """The residual-VJP kernel alone on the n^2 p = 3 FP32 vortex (1024^2:
    268 MB per state array, above L2): mean time of `reps` launches after one
    untimed launch, against its algorithmic bytes (reads q and the cotangent,
    writes the result: 3 state arrays, 48 B per DOF)."""
    import torch
    from paper_1709_01619_gb300 import _native as nat
    from paper_1709_01619_gb300 import inputs
    c = nat.Config(eqn=nat.EULER, nx=n, ny=n, p=3, x1=L, y1=L, dtype=nat.F32)
    with nat.Context(c) as cx:
        x, y = cx.point_coords()
        q = torch.tensor(inputs.vortex(x, y, eps=EPS), dtype=torch.float32, device="cuda")
        rbar = torch.tensor(inputs.noise(tuple(q.shape), 11, 1.0), dtype=torch.float32, device="cuda")
        qbar = torch.empty_like(q)
        cx.residual_vjp(q, rbar, qbar)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            cx.residual_vjp(q, rbar, qbar)
        e1.record()
        torch.cuda.synchronize()
        launch = e0.elapsed_time(e1) / reps
    achieved = n * n * 16 * 48 / (launch * 1e-3) / 1e9
    return {"workload": f"euler_vortex_{n}x{n}_p3_fp32_residual_vjp", "launch_ms": launch, "bound": "hbm",
            "bytes_per_dof": 48, "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak}


def adjoint_case(peak):
    """Gradient of J = 1/2 sum W (q_N - q_t)^2 with respect to the initial
    state: Euler vortex (strength 5) on [0,10]^2, 256^2, p = 3, FP32, 400
    SSP-RK3 steps of dt = 7e-4 (t = 0.28, CFL 0.07), checkpoints every 20
    steps, q_t the forward solution from strength 4.5.  Forward (with
    checkpoints) and backward (recompute + transposed steps) timed with CUDA
    events.  The residual-VJP kernel alone: mean launch time at 256^2 and on
    the 1024^2 vortex (268 MB per array, above L2), against its algorithmic
    bytes (it reads q and the cotangent and writes the result: 3 state
    arrays, 48 B per DOF in FP32)."""
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
    vjp = {f"{m}": vjp_case(peak, 50 if m == 256 else 10, m) for m in (256, 1024)}
    return {"workload": "euler_vortex_256x256_p3_fp32_adjoint_400steps_ckpt20", "forward_ms": fwd,
            "backward_ms": bwd, "gradient_ms": fwd + bwd, "backward_over_forward": bwd / fwd,
            "forward_dof_stage_per_s": dof * 3 * nsteps / (fwd * 1e-3), "gradient_finite": finite,
            "vjp_kernel": {"bound": "hbm", "bytes_per_dof": 48, "peak": peak, "unit": "GB/s", **vjp}}


def run_cpr(args, world, rank, local):
    peak, peak_kind = peaks()
    head = batch_headline(args, world, local, peak)
    cfg = {"workload": WORKLOAD, "instances": BATCH_N, "seed": BATCH_SEED,
           "N": "U{32..256}", "p": "U{2,3,4}", "strength": "U[1,5]", "dof": head["dof"],
           "rk3_steps_per_pass": BATCH_STEPS, "cfl": "0.1/0.06/0.04 (p=2/3/4)", "points": "gauss",
           "flux": "rusanov", "form": "per-instance chains" if head["per_instance"] else "grouped launches",
           "l2_flush": "inputs larger than L2 (445 MB per state array; states reset before each pass, "
                       "outside the timed events)", "replicas": world}
    line = {
        "metric": METRIC, "value": head["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": head["ms_max"] / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic", "config": cfg,
        "roofline": {**head["roofline"], "peak_source": peak_kind},
        "e2e": {"value": head["e2e"], "unit": UNIT, "h2d_bytes_per_step": head["state_bytes"],
                "d2h_bytes_per_step": head["state_bytes"]},
        "gpu_launches": head["gpu_launches"], "clocks": head["clocks"],
    }
    detail = {"headline": {k: head[k] for k in ("tuned", "per_instance", "steps_done", "t_min", "t_max",
                                                "finite", "e2e_equal", "clocks_e2e")}}
    if args.quick:
        if rank == 0:
            print(json.dumps(compact(line)), flush=True)
        return
    import torch

    def mk(dtype, nx, p=P):
        return make_vortex(dtype, nx, p)

    side = {}
    side["hbm1024"] = hbm_case(mk, peak)
    v128 = vortex128_case(peak)
    side["vortex128"] = v128
    side["equal_error"] = equal_error_case(v128)
    side["limited"] = limited_case(peak)
    fv = fv_case(peak)
    fv["cpr_512_p2_over_fv_time_to_solution"] = side["limited"]["ms_fp32"] / fv["ms_fp32"]
    side["fv_equal_dof"] = fv
    side["radial_shock_tube"] = radial_case()
    side["adjoint"] = adjoint_case(peak)
    side["paper_setting"] = paper_setting_case()
    torch.cuda.synchronize()
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        states = oracle_batch_states()
        v, work, secs, thr = oracle_batch_sample(1, states=states)
        sub = states[::4]
        v1, work1, secs1, _ = oracle_batch_sample(1, threads=1, states=sub)
        cpu = {"value": v, "unit": UNIT, "cores": thr, "kind": "oracle",
               "sample": f"1 FP64 SSP-RK3 CFL step of all 64 instances ({work:.3g} DOF-stages, {secs:.1f} s)",
               "single_thread": {"value": v1, "sample": f"1 step of every 4th instance ({secs1:.1f} s)"},
               "cpu": cpu_model()}
    line["cpu_baseline"] = cpu
    if rank != 0:
        return
    h, v, e, lim, fvq, rad, adj = (side["hbm1024"], side["vortex128"], side["equal_error"], side["limited"],
                                   side["fv_equal_dof"], side["radial_shock_tube"], side["adjoint"])
    # compact side blocks on the line itself; full records on stderr
    line["hbm1024"] = {"frac": h["frac"], "moved_frac": h["moved_frac"], "launch_ms": h["launch_ms"],
                       "traffic": h["traffic"], "rate": h["dof_stage_per_s"]}
    line["vortex128"] = {"f32_rate": v["dof_stage_per_s_fp32"], "f64_rate": v["dof_stage_per_s_fp64"],
                         "same_grid_f32_over_f64": v["same_grid_f32_over_f64"],
                         "err_f32": v["l2_rho_avg_error"]["f32"], "err_f64": v["l2_rho_avg_error"]["f64"],
                         "f32_vs_f64": v["f32_vs_f64_rel_l2"], "frac": v["roofline"]["frac"],
                         "f64_alu_frac": v["f64_roofline"]["frac"],
                         "f64_alu_frac_executed": v["f64_roofline"]["executed_frac"]}
    fr = e["frontier"]
    line["equal_error_speedup"] = {
        "error": e["f32_128_run"]["error"],
        "f32_128_run_vs_f64_interp": e["f32_128_run"]["speedup_f32_over_f64"],
        "frontier_at_f32_128_error": fr[f"{e['f32_128_run']['error']:.3g}"]["speedup_f32_over_f64"],
        "frontier_at_1e-6": fr["1e-06"]["speedup_f32_over_f64"],
        "frontier_at_3e-6": fr["3e-06"]["speedup_f32_over_f64"]}
    line["limited"] = {"ms_f32": lim["ms_fp32"], "rate_f32": lim["dof_stage_per_s_fp32"], "frac": lim["frac"],
                       "rate_f64": lim["dof_stage_per_s_fp64"], "f32_vs_f64": lim.get("f32_vs_f64_rel_l2")}
    line["fv"] = {"ms_muscl2": fvq["ms_fp32"], "ms_muscl3": fvq["muscl3"]["ms_fp32"],
                  "cpr_over_fv_time": fvq["cpr_512_p2_over_fv_time_to_solution"]}
    line["radial"] = {"cpr_ms": rad["cpr_400_p2"]["ms"], "fv2_ms": rad["fv_muscl2_1200"]["ms"],
                      "fv3_ms": rad["fv_muscl3_1200"]["ms"]}
    line["adjoint"] = {"fwd_ms": adj["forward_ms"], "bwd_ms": adj["backward_ms"],
                       "vjp_frac_1024": adj["vjp_kernel"]["1024"]["frac"],
                       "vjp_ms_256": adj["vjp_kernel"]["256"]["launch_ms"]}
    line["paper_setting"] = {"rate": side["paper_setting"]["dof_stage_per_s"],
                             "err": side["paper_setting"]["l2_rho_avg_error"]}
    detail.update(side)
    detail["cpu_baseline"] = cpu
    print(json.dumps(compact(detail, 6)), file=sys.stderr, flush=True)
    print(json.dumps(compact(line)), flush=True)


def run_block(args):
    """--workload other than headline: one block alone (profiling runs)."""
    peak, _ = peaks()
    w = args.workload
    if w == "vortex1024":
        out = hbm_case(make_vortex, peak, max(1, args.steps), args.p)
    elif w == "batch":
        out = batch_case(peak, steps=max(1, args.steps), warmup=args.warmup, tune=not args.no_tune,
                         per_instance=args.per_instance)
    elif w == "limited":
        out = limited_case(peak, fp64_steps=max(1, args.steps))
    elif w == "radial":
        out = radial_case()
    elif w == "fv1536":
        out = fv_case(peak, fp64_steps=max(1, args.steps))
    elif w == "vortex128":
        out = vortex128_case(peak)
    elif w == "ladder":
        out = equal_error_case(vortex128_case(peak))
    elif w == "adjoint":
        out = adjoint_case(peak)
    elif w == "vjp":
        out = vjp_case(peak, max(1, args.steps))
    else:  # f64
        out = run_f64_only(args)
    print(json.dumps(compact(out, 6)), flush=True)


def run_f64_only(args):
    """FP64 path on the 128^2 p = 3 vortex: `steps` CFL RK3 steps timed after
    three untimed ones (a short run for profiling the FP64 stage kernel)."""
    import torch
    from paper_1709_01619_gb300 import _native as nat
    cfg, ctx, q = make_vortex(nat.F64, NX, P)
    with ctx:
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
    return {"workload": "euler_vortex_128x128_p3_fp64", "rk3_steps": args.steps, "ms": ms,
            "dof_stage_per_s": rate, **f64_roofline(rate)}


def main():
    args = parse()
    world, rank, local = dist_setup()
    if args.impl == "reference":
        run_reference(args, world, rank)
    elif args.workload == "headline":
        run_cpr(args, world, rank, local)
    else:
        run_block(args)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
