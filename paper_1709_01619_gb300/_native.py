"""ctypes binding of libcpr.so (include/cpr.h).

Argument marshalling only: every step of the CPR path runs in the library's
CUDA kernels.  PyTorch supplies device memory and the current stream.  The
library is built in-tree by :mod:`paper_1709_01619_gb300.build`; if it cannot
be built or loaded, every call raises -- there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import dataclasses
import os
import threading

import torch

from . import build as _build

CPR_OK, CPR_EINVAL, CPR_ENOMEM, CPR_ECUDA, CPR_ENONPHYS, CPR_ETIMEOUT, CPR_ENOTIMPL = range(7)
ADVECTION, EULER = 0, 1
GAUSS, LOBATTO = 0, 1
CORR_GDG, CORR_NDG, CORR_NDG_LUMPED = 0, 1, 2
RUSANOV, UPWIND, ROE = 0, 1, 2
DIV_LP, DIV_CHAIN = 0, 1
PERIODIC, TRANSMISSIVE = 0, 1
F64, F32 = 0, 1
SCHEME_CPR, SCHEME_FV_MUSCL, SCHEME_FV_MUSCL3 = 0, 1, 2

_STATUS = {0: "CPR_OK", 1: "CPR_EINVAL", 2: "CPR_ENOMEM", 3: "CPR_ECUDA", 4: "CPR_ENONPHYS",
           5: "CPR_ETIMEOUT", 6: "CPR_ENOTIMPL"}

# every entry point declared in include/cpr.h
EXPORTS = (
    "cpr_init", "cpr_destroy", "cpr_state_elems", "cpr_last_error", "cpr_point_coords",
    "cpr_residual", "cpr_step", "cpr_step_host", "cpr_limit", "cpr_get_marks", "cpr_averages",
    "cpr_norms", "cpr_set_time", "cpr_get_time", "cpr_residual_vjp", "cpr_step_vjp",
    "cpr_step_stages", "cpr_step_vjp_stages",
    "cpr_step_noalloc", "cpr_batch_init", "cpr_batch_destroy", "cpr_batch_last_error",
    "cpr_batch_step", "cpr_batch_step_host", "cpr_batch_tune", "cpr_batch_set_form", "cpr_batch_get_time",
    "cpr_batch_set_time",
)


class CprError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{_STATUS.get(status, status)}: {msg}")
        self.status = status


class _Config(ctypes.Structure):
    _fields_ = [
        ("eqn", ctypes.c_int), ("nx", ctypes.c_int), ("ny", ctypes.c_int),
        ("x0", ctypes.c_double), ("x1", ctypes.c_double), ("y0", ctypes.c_double),
        ("y1", ctypes.c_double), ("p", ctypes.c_int), ("pts", ctypes.c_int),
        ("corr", ctypes.c_int), ("flux", ctypes.c_int), ("div", ctypes.c_int),
        ("ax", ctypes.c_double), ("ay", ctypes.c_double), ("gamma", ctypes.c_double),
        ("bc_x", ctypes.c_int), ("bc_y", ctypes.c_int), ("limiter", ctypes.c_int),
        ("tvb_M", ctypes.c_double), ("lim_eps", ctypes.c_double), ("dtype", ctypes.c_int),
        ("cfl", ctypes.c_double), ("scheme", ctypes.c_int),
    ]


class _Norms(ctypes.Structure):
    _fields_ = [
        ("sum_avg", ctypes.c_double * 4), ("l2_abs", ctypes.c_double),
        ("l2_rel", ctypes.c_double), ("max_wave", ctypes.c_double),
        ("n_nonphys", ctypes.c_longlong), ("n_marked", ctypes.c_longlong),
        ("t", ctypes.c_double), ("steps", ctypes.c_longlong),
    ]


@dataclasses.dataclass
class Config:
    """Mirror of ``cpr_config``."""
    eqn: int = EULER
    nx: int = 16
    ny: int = 16
    x0: float = 0.0
    x1: float = 1.0
    y0: float = 0.0
    y1: float = 1.0
    p: int = 2
    pts: int = GAUSS
    corr: int = CORR_GDG
    flux: int = RUSANOV
    div: int = DIV_LP
    ax: float = 1.0
    ay: float = 1.0
    gamma: float = 1.4
    bc_x: int = PERIODIC
    bc_y: int = PERIODIC
    limiter: int = 0
    tvb_M: float = 0.0
    lim_eps: float = 1e-3
    dtype: int = F64
    cfl: float = 0.1
    scheme: int = 0  # SCHEME_CPR, or SCHEME_FV_MUSCL / SCHEME_FV_MUSCL3 (p = 0: one average per element)

    @property
    def nvars(self) -> int:
        return 4 if self.eqn == EULER else 1

    @property
    def ne(self) -> int:
        return self.nx * self.ny

    @property
    def shape(self):
        return (self.nvars, self.ne, (self.p + 1) ** 2)

    @property
    def torch_dtype(self):
        return torch.float32 if self.dtype == F32 else torch.float64

    def _c(self) -> _Config:
        return _Config(**dataclasses.asdict(self))


_lock = threading.Lock()
_lib = None


def library_path() -> str:
    return _build.LIB


def load():
    """Load libcpr.so, building it first when it is missing or stale."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.build()
            if not os.path.exists(path):
                raise RuntimeError("libcpr.so is missing and could not be built")
            lib = ctypes.CDLL(path)
            P, I, D, LL = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_longlong
            lib.cpr_init.restype = I
            lib.cpr_init.argtypes = [ctypes.POINTER(_Config), P, ctypes.POINTER(P)]
            lib.cpr_destroy.restype = None
            lib.cpr_destroy.argtypes = [P]
            lib.cpr_state_elems.restype = ctypes.c_size_t
            lib.cpr_state_elems.argtypes = [P]
            lib.cpr_last_error.restype = ctypes.c_char_p
            lib.cpr_last_error.argtypes = [P]
            lib.cpr_point_coords.restype = I
            lib.cpr_point_coords.argtypes = [P, P, P]
            lib.cpr_residual.restype = I
            lib.cpr_residual.argtypes = [P, P, P]
            lib.cpr_step.restype = I
            lib.cpr_step.argtypes = [P, P, I, D, D]
            lib.cpr_step_host.restype = I
            lib.cpr_step_host.argtypes = [P, P, P, I, D, D]
            lib.cpr_limit.restype = I
            lib.cpr_limit.argtypes = [P, P]
            lib.cpr_get_marks.restype = I
            lib.cpr_get_marks.argtypes = [P, P]
            lib.cpr_averages.restype = I
            lib.cpr_averages.argtypes = [P, P, P]
            lib.cpr_norms.restype = I
            lib.cpr_norms.argtypes = [P, P, P, ctypes.POINTER(_Norms)]
            lib.cpr_set_time.restype = I
            lib.cpr_set_time.argtypes = [P, D, LL]
            lib.cpr_get_time.restype = I
            lib.cpr_get_time.argtypes = [P, ctypes.POINTER(D), ctypes.POINTER(LL)]
            lib.cpr_residual_vjp.restype = I
            lib.cpr_residual_vjp.argtypes = [P, P, P, P]
            lib.cpr_step_vjp.restype = I
            lib.cpr_step_vjp.argtypes = [P, P, P, P, D]
            lib.cpr_step_stages.restype = I
            lib.cpr_step_stages.argtypes = [P, P, P, P, P, D]
            lib.cpr_step_vjp_stages.restype = I
            lib.cpr_step_vjp_stages.argtypes = [P, P, P, P, P, P, D]
            lib.cpr_batch_init.restype = I
            lib.cpr_batch_init.argtypes = [ctypes.POINTER(_Config), I, P, ctypes.POINTER(P)]
            lib.cpr_batch_destroy.restype = None
            lib.cpr_batch_destroy.argtypes = [P]
            lib.cpr_batch_last_error.restype = ctypes.c_char_p
            lib.cpr_batch_last_error.argtypes = [P]
            lib.cpr_batch_step.restype = I
            lib.cpr_batch_step.argtypes = [P, ctypes.POINTER(P), I, D, D]
            lib.cpr_batch_step_host.restype = I
            lib.cpr_batch_step_host.argtypes = [P, ctypes.POINTER(P), ctypes.POINTER(P), I, D, D]
            lib.cpr_batch_tune.restype = I
            lib.cpr_batch_tune.argtypes = [P, ctypes.POINTER(P), ctypes.POINTER(I), ctypes.POINTER(I)]
            lib.cpr_batch_set_form.restype = I
            lib.cpr_batch_set_form.argtypes = [P, I]
            lib.cpr_batch_get_time.restype = I
            lib.cpr_batch_get_time.argtypes = [P, I, ctypes.POINTER(D), ctypes.POINTER(LL)]
            lib.cpr_batch_set_time.restype = I
            lib.cpr_batch_set_time.argtypes = [P, D, LL]
            _lib = lib
    return _lib


def _ptr(t):
    if t is None:
        return None
    return ctypes.c_void_p(t.data_ptr())


class Context:
    """One CPR problem on the current CUDA device (wraps ``cpr_ctx``)."""

    def __init__(self, cfg: Config, stream=None):
        if not torch.cuda.is_available():
            raise RuntimeError("the CPR kernels need a CUDA device")
        self.lib = load()
        self.cfg = cfg
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        h = ctypes.c_void_p()
        st = self.lib.cpr_init(ctypes.byref(cfg._c()), ctypes.c_void_p(stream.cuda_stream), ctypes.byref(h))
        if st != CPR_OK:
            raise CprError(st, self.lib.cpr_last_error(None).decode())
        self.h = h

    # -- helpers -------------------------------------------------------------
    def _check(self, st):
        if st != CPR_OK:
            raise CprError(st, self.lib.cpr_last_error(self.h).decode())

    def _state(self, t, name="q"):
        if not isinstance(t, torch.Tensor):
            raise TypeError(f"{name} must be a torch.Tensor")
        if t.device.type != "cuda":
            raise ValueError(f"{name} must live on a CUDA device")
        if t.dtype != self.cfg.torch_dtype:
            raise ValueError(f"{name} must be {self.cfg.torch_dtype}")
        if not t.is_contiguous() or t.numel() != self.state_elems:
            raise ValueError(f"{name} must be contiguous with {self.state_elems} values")
        return t

    @property
    def state_elems(self) -> int:
        return int(self.lib.cpr_state_elems(self.h))

    def empty_state(self):
        return torch.empty(self.cfg.shape, dtype=self.cfg.torch_dtype, device="cuda")

    # -- entry points ----------------------------------------------------------
    def point_coords(self):
        import numpy as np
        x = np.empty((self.cfg.ne, (self.cfg.p + 1) ** 2))
        y = np.empty_like(x)
        self._check(self.lib.cpr_point_coords(self.h, x.ctypes.data_as(ctypes.c_void_p),
                                              y.ctypes.data_as(ctypes.c_void_p)))
        return x, y

    def residual(self, q, r=None):
        self._state(q)
        if r is None:
            r = torch.empty_like(q)
        self._state(r, "r")
        self._check(self.lib.cpr_residual(self.h, _ptr(q), _ptr(r)))
        return r

    def step(self, q, nsteps: int, dt_fixed: float = 0.0, t_end: float = 0.0):
        self._state(q)
        self._check(self.lib.cpr_step(self.h, _ptr(q), int(nsteps), float(dt_fixed), float(t_end)))
        return q

    def step_host(self, q_in, q_out=None, nsteps: int = 1, dt_fixed: float = 0.0, t_end: float = 0.0):
        if q_out is None:
            q_out = q_in
        for t, n in ((q_in, "q_in"), (q_out, "q_out")):
            if t.device.type != "cpu" or t.dtype != self.cfg.torch_dtype or not t.is_contiguous() \
                    or t.numel() != self.state_elems:
                raise ValueError(f"{n} must be a contiguous host tensor of the state size")
        self._check(self.lib.cpr_step_host(self.h, _ptr(q_in), _ptr(q_out), int(nsteps),
                                           float(dt_fixed), float(t_end)))
        return q_out

    def limit(self, q):
        self._state(q)
        self._check(self.lib.cpr_limit(self.h, _ptr(q)))
        return q

    def get_marks(self):
        import numpy as np
        m = np.empty(self.cfg.ne, dtype=np.int32)
        self._check(self.lib.cpr_get_marks(self.h, m.ctypes.data_as(ctypes.c_void_p)))
        return m

    def averages(self, q):
        self._state(q)
        avg = torch.empty((self.cfg.nvars, self.cfg.ne), dtype=q.dtype, device=q.device)
        self._check(self.lib.cpr_averages(self.h, _ptr(q), _ptr(avg)))
        return avg

    def norms(self, q, ref=None) -> dict:
        self._state(q)
        if ref is not None:
            self._state(ref, "ref")
        out = _Norms()
        st = self.lib.cpr_norms(self.h, _ptr(q), _ptr(ref), ctypes.byref(out))
        if st not in (CPR_OK, CPR_ENONPHYS):
            self._check(st)
        return {"sum_avg": list(out.sum_avg[:self.cfg.nvars]), "l2_abs": out.l2_abs,
                "l2_rel": out.l2_rel, "max_wave": out.max_wave, "n_nonphys": out.n_nonphys,
                "n_marked": out.n_marked, "t": out.t, "steps": out.steps, "status": st}

    def set_time(self, t: float, steps: int = 0):
        self._check(self.lib.cpr_set_time(self.h, float(t), int(steps)))

    def get_time(self):
        t = ctypes.c_double()
        s = ctypes.c_longlong()
        self._check(self.lib.cpr_get_time(self.h, ctypes.byref(t), ctypes.byref(s)))
        return t.value, s.value

    def residual_vjp(self, q, rbar, qbar=None):
        self._state(q)
        self._state(rbar, "rbar")
        if qbar is None:
            qbar = torch.empty_like(q)
        self._check(self.lib.cpr_residual_vjp(self.h, _ptr(q), _ptr(rbar), _ptr(qbar)))
        return qbar

    def step_vjp(self, q, qbar_out, dt: float, qbar_in=None):
        self._state(q)
        self._state(qbar_out, "qbar_out")
        if qbar_in is None:
            qbar_in = torch.empty_like(q)
        self._check(self.lib.cpr_step_vjp(self.h, _ptr(q), _ptr(qbar_out), _ptr(qbar_in), float(dt)))
        return qbar_in

    def step_stages(self, q, q1, q2, q_next, dt: float):
        """One Shu-Osher SSP-RK3 step of size dt from q into q_next, keeping
        the stage states q1, q2 (cpr_step_stages)."""
        for t, n in ((q, "q"), (q1, "q1"), (q2, "q2"), (q_next, "q_next")):
            self._state(t, n)
        self._check(self.lib.cpr_step_stages(self.h, _ptr(q), _ptr(q1), _ptr(q2), _ptr(q_next), float(dt)))
        return q_next

    def step_vjp_stages(self, q, q1, q2, qbar_out, dt: float, qbar_in=None):
        """cpr_step_vjp around the given stage states (cpr_step_vjp_stages)."""
        for t, n in ((q, "q"), (q1, "q1"), (q2, "q2"), (qbar_out, "qbar_out")):
            self._state(t, n)
        if qbar_in is None:
            qbar_in = torch.empty_like(q)
        self._check(self.lib.cpr_step_vjp_stages(self.h, _ptr(q), _ptr(q1), _ptr(q2), _ptr(qbar_out),
                                                 _ptr(qbar_in), float(dt)))
        return qbar_in

    def close(self):
        if getattr(self, "h", None):
            self.lib.cpr_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


class Batch:
    """Many CPR problems advanced together (wraps ``cpr_batch``)."""

    def __init__(self, cfgs, stream=None):
        if not torch.cuda.is_available():
            raise RuntimeError("the CPR kernels need a CUDA device")
        self.lib = load()
        self.cfgs = list(cfgs)
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        arr = (_Config * len(self.cfgs))(*[c._c() for c in self.cfgs])
        h = ctypes.c_void_p()
        st = self.lib.cpr_batch_init(arr, len(self.cfgs), ctypes.c_void_p(stream.cuda_stream), ctypes.byref(h))
        if st != CPR_OK:
            raise CprError(st, self.lib.cpr_batch_last_error(None).decode())
        self.h = h

    def _check(self, st):
        if st != CPR_OK:
            raise CprError(st, self.lib.cpr_batch_last_error(self.h).decode())

    def _ptrs(self, qs):
        if len(qs) != len(self.cfgs):
            raise ValueError("one state per instance")
        for q, c in zip(qs, self.cfgs):
            if q.device.type != "cuda" or q.dtype != c.torch_dtype or not q.is_contiguous() \
                    or q.numel() != c.nvars * c.ne * (c.p + 1) ** 2:
                raise ValueError("each state must be a contiguous CUDA tensor of its instance's size")
        return (ctypes.c_void_p * len(qs))(*[q.data_ptr() for q in qs])

    def empty_states(self):
        return [torch.empty(c.shape, dtype=c.torch_dtype, device="cuda") for c in self.cfgs]

    def step(self, qs, nsteps: int, dt_fixed: float = 0.0, t_end: float = 0.0):
        self._check(self.lib.cpr_batch_step(self.h, self._ptrs(qs), int(nsteps), float(dt_fixed),
                                            float(t_end)))
        return qs

    def step_host(self, qs_in, qs_out=None, nsteps: int = 1, dt_fixed: float = 0.0, t_end: float = 0.0):
        """cpr_batch_step on host (preferably pinned) tensors: copies in,
        steps, copies out, synchronises."""
        if qs_out is None:
            qs_out = qs_in
        if len(qs_in) != len(self.cfgs) or len(qs_out) != len(self.cfgs):
            raise ValueError("one state per instance")
        for group in (qs_in, qs_out):
            for q, c in zip(group, self.cfgs):
                if q.device.type != "cpu" or q.dtype != c.torch_dtype or not q.is_contiguous() \
                        or q.numel() != c.nvars * c.ne * (c.p + 1) ** 2:
                    raise ValueError("each state must be a contiguous host tensor of its instance's size")
        pin = (ctypes.c_void_p * len(qs_in))(*[q.data_ptr() for q in qs_in])
        pout = (ctypes.c_void_p * len(qs_out))(*[q.data_ptr() for q in qs_out])
        self._check(self.lib.cpr_batch_step_host(self.h, pin, pout, int(nsteps), float(dt_fixed), float(t_end)))
        return qs_out

    def tune(self, qs):
        choices = (ctypes.c_int * 12)()
        ng = ctypes.c_int()
        self._check(self.lib.cpr_batch_tune(self.h, self._ptrs(qs), choices, ctypes.byref(ng)))
        return [tuple(choices[3 * k:3 * k + 3]) for k in range(ng.value)]

    def set_form(self, per_instance: bool):
        """Grouped launches (False) or per-instance launch chains (True)."""
        self._check(self.lib.cpr_batch_set_form(self.h, int(bool(per_instance))))

    def get_time(self, i: int):
        t = ctypes.c_double()
        s = ctypes.c_longlong()
        self._check(self.lib.cpr_batch_get_time(self.h, int(i), ctypes.byref(t), ctypes.byref(s)))
        return t.value, s.value

    def set_time(self, t: float, steps: int = 0):
        self._check(self.lib.cpr_batch_set_time(self.h, float(t), int(steps)))

    def close(self):
        if getattr(self, "h", None):
            self.lib.cpr_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
