"""cpr_step_noalloc: the fixed-step RK3 entry point that allocates nothing.

It exists for callers that cannot let a library allocate device memory (a
host framework whose pool allocator owns the device, or a loop where the
device synchronisation of cudaMalloc is not allowed).  Its stage buffers live
in a fixed device array inside libcpr.so.  Checked here through the C ABI
against cpr_step (the context-based entry point) on two calls in a row, and
for its size limit.  Collected last on purpose, and independent of the other
tests' state.
"""
import ctypes

import numpy as np
import pytest
import torch

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
    a, b = a.double().cpu().numpy(), b.double().cpu().numpy()
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.mark.parametrize("dtype", [nat.F64, nat.F32])
@pytest.mark.parametrize("eqn", [nat.EULER, nat.ADVECTION])
def test_noalloc_matches_cpr_step_on_two_calls(dtype, eqn):
    lib = _lib()
    cfg = nat.Config(eqn=eqn, nx=21, ny=17, p=3, x1=10.0, y1=8.0, dtype=dtype,
                     flux=nat.RUSANOV, ax=0.9, ay=-0.4)
    dt, n = 2e-3, 4
    stream = torch.cuda.current_stream()
    with nat.Context(cfg, stream) as ctx:
        x, y = ctx.point_coords()
        q0 = inputs.vortex(x, y, eps=4.0, xc=5.0, yc=4.0, ly=8.0)
        if eqn == nat.ADVECTION:
            q0 = q0[:1]
        ref = torch.tensor(q0, dtype=cfg.torch_dtype, device="cuda")
        mine = ref.clone()
        for call in range(2):
            ctx.step(ref, n, dt)
            st = lib.cpr_step_noalloc(ctypes.byref(cfg._c()), ctypes.c_void_p(mine.data_ptr()), n, dt,
                                      ctypes.c_void_p(stream.cuda_stream))
            assert st == nat.CPR_OK, f"call {call}: status {st}"
            torch.cuda.synchronize()
            assert _rel(mine, ref) <= TOL[dtype], f"call {call}"


def test_noalloc_rejects_states_beyond_its_scratch():
    lib = _lib()
    # 512 x 512 elements, p = 2, FP32 Euler: 37.7 MB > 16 MiB
    cfg = nat.Config(eqn=nat.EULER, nx=512, ny=512, p=2, dtype=nat.F32)
    q = torch.zeros(16, dtype=torch.float32, device="cuda")
    st = lib.cpr_step_noalloc(ctypes.byref(cfg._c()), ctypes.c_void_p(q.data_ptr()), 1, 1e-3, None)
    assert st == nat.CPR_EINVAL
    cfg = nat.Config(eqn=nat.EULER, nx=8, ny=8, p=2, limiter=1)
    assert lib.cpr_step_noalloc(ctypes.byref(cfg._c()), ctypes.c_void_p(q.data_ptr()), 1, 1e-3,
                                None) == nat.CPR_EINVAL
