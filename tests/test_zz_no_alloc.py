"""cpr_step_noalloc: the fixed-step RK3 entry point that allocates nothing.

It exists for callers that cannot let a library allocate device memory (a
host framework whose pool allocator owns the device, or a loop where the
device synchronisation of cudaMalloc is not allowed).  Its stage buffers and
the low part of the FP32 state live in a fixed device array inside
libcpr.so.  Checked here through the C ABI against cpr_step (the
context-based entry point) on two calls in a row, against the FP64 oracle
(a few steps, and a few hundred FP32 steps), and for its argument rules.
Collected last on purpose, and independent of the other tests' state.
"""
import ctypes
import math

import numpy as np
import pytest
import torch

import oracle
from paper_1709_01619_gb300 import _native as nat
from paper_1709_01619_gb300 import inputs

pytestmark = pytest.mark.gpu

TOL = {nat.F64: 1e-12, nat.F32: 1e-5}


def _lib():
    lib = nat.load()
    lib.cpr_step_noalloc.restype = ctypes.c_int
    lib.cpr_step_noalloc.argtypes = [ctypes.POINTER(nat._Config), ctypes.c_void_p, ctypes.c_int,
                                     ctypes.c_double, ctypes.c_void_p]
    return lib


def _rel(a, b):
    a = a.double().cpu().numpy() if torch.is_tensor(a) else np.asarray(a)
    b = b.double().cpu().numpy() if torch.is_tensor(b) else np.asarray(b)
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def _vortex_case(eqn, dtype, nx=21, ny=17, p=3):
    cfg = nat.Config(eqn=eqn, nx=nx, ny=ny, p=p, x1=10.0, y1=8.0, dtype=dtype,
                     flux=nat.RUSANOV, ax=0.9, ay=-0.4)
    o = oracle.Config(eqn=eqn, nx=nx, ny=ny, p=p, x1=10.0, y1=8.0, flux=oracle.RUSANOV, ax=0.9, ay=-0.4)
    x, y = oracle.point_coords(o)
    q0 = inputs.vortex(x, y, eps=4.0, xc=5.0, yc=4.0, ly=8.0)
    if eqn == nat.ADVECTION:
        q0 = q0[:1]
    if dtype == nat.F32:
        q0 = q0.astype(np.float32).astype(np.float64)
    return cfg, o, q0


def _noalloc(lib, cfg, q, n, dt, stream=None):
    s = ctypes.c_void_p(stream.cuda_stream) if stream is not None else None
    return lib.cpr_step_noalloc(ctypes.byref(cfg._c()), ctypes.c_void_p(q.data_ptr()), n, dt, s)


@pytest.mark.parametrize("dtype", [nat.F64, nat.F32])
@pytest.mark.parametrize("eqn", [nat.EULER, nat.ADVECTION])
def test_noalloc_matches_cpr_step_on_two_calls(dtype, eqn):
    """Two calls in a row (odd step counts, so the FP32 high part ends in
    the scratch array and is copied back) against cpr_step stepping a copy
    of the same state."""
    lib = _lib()
    cfg, _, q0 = _vortex_case(eqn, dtype)
    dt, n = 2e-3, 3
    stream = torch.cuda.current_stream()
    with nat.Context(cfg, stream) as ctx:
        ref = torch.tensor(q0.reshape(cfg.shape), dtype=cfg.torch_dtype, device="cuda")
        mine = ref.clone()
        for call in range(2):
            ctx.step(ref, n, dt)
            st = _noalloc(lib, cfg, mine, n, dt, stream)
            assert st == nat.CPR_OK, f"call {call}: status {st}"
            torch.cuda.synchronize()
            assert _rel(mine, ref) <= TOL[dtype], f"call {call}"


@pytest.mark.parametrize("dtype", [nat.F64, nat.F32])
@pytest.mark.parametrize("eqn", [nat.EULER, nat.ADVECTION])
def test_noalloc_matches_oracle(dtype, eqn):
    lib = _lib()
    cfg, o, q0 = _vortex_case(eqn, dtype)
    dt, n = 2e-3, 4
    q_or, _, _ = oracle.run(o, q0, n, dt)
    q = torch.tensor(q0.reshape(cfg.shape), dtype=cfg.torch_dtype, device="cuda")
    assert _noalloc(lib, cfg, q, n, dt) == nat.CPR_OK
    torch.cuda.synchronize()
    assert _rel(q, q_or) <= TOL[dtype]


def test_noalloc_fp32_long_run_vs_oracle():
    """300 FP32 steps (t = 3, about 0.6 of the CFL limit) of the vortex on
    16 x 16 p = 3 elements in calls of 100 steps: the compensated form keeps
    the state within the FP32 tolerance of the FP64 oracle."""
    lib = _lib()
    cfg, o, q0 = _vortex_case(nat.EULER, nat.F32, nx=16, ny=16)
    dt = 0.01
    q_or, _, _ = oracle.run(o, q0, 300, dt)
    q = torch.tensor(q0.reshape(cfg.shape), dtype=torch.float32, device="cuda")
    for _ in range(3):
        assert _noalloc(lib, cfg, q, 100, dt) == nat.CPR_OK
    torch.cuda.synchronize()
    assert _rel(q, q_or) <= TOL[nat.F32]


def test_noalloc_argument_rules():
    """Sizes beyond the fixed scratch, the limiter, the FV schemes and any
    configuration cpr_init rejects (a non-finite domain bound, a bad flux
    for the equation) return CPR_EINVAL before any work; Roe's flux, which
    cpr_init accepts, is accepted."""
    lib = _lib()
    q = torch.zeros(8 * 8 * 9 * 4, dtype=torch.float64, device="cuda")
    # 512 x 512 elements, p = 2, FP32 Euler: 37.7 MB > 16 MiB
    big = nat.Config(eqn=nat.EULER, nx=512, ny=512, p=2, dtype=nat.F32)
    assert _noalloc(lib, big, q, 1, 1e-3) == nat.CPR_EINVAL
    bad = [
        nat.Config(eqn=nat.EULER, nx=8, ny=8, p=2, limiter=1),
        nat.Config(eqn=nat.EULER, nx=8, ny=8, p=0, scheme=nat.SCHEME_FV_MUSCL),
        nat.Config(eqn=nat.EULER, nx=8, ny=8, p=2, x1=math.inf),
        nat.Config(eqn=nat.EULER, nx=8, ny=8, p=2, flux=nat.UPWIND),
        nat.Config(eqn=nat.EULER, nx=8, ny=8, p=5),
    ]
    for c in bad:
        assert _noalloc(lib, c, q, 1, 1e-3) == nat.CPR_EINVAL, c
    ok = nat.Config(eqn=nat.EULER, nx=8, ny=8, p=2, flux=nat.ROE)
    q.copy_(torch.tensor(_vortex_case(nat.EULER, nat.F64, 8, 8, 2)[2].ravel()))
    assert _noalloc(lib, ok, q, 1, 1e-3) == nat.CPR_OK
    torch.cuda.synchronize()
    assert bool(torch.isfinite(q).all())
    assert _noalloc(lib, ok, q, 1, -1.0) == nat.CPR_EINVAL
