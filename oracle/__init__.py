"""FP64 CPU oracle of the CPR hot path (arXiv 1709.01619), numpy front end.

TEST INFRASTRUCTURE ONLY.  The tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` are the only callers.  The arithmetic lives in
``cpr_oracle.c`` (plain C, double precision, built with -ffp-contract=off); this
module compiles it on demand and marshals numpy arrays.  It imports nothing
from the CUDA package and the CUDA package imports nothing from here.

State layout: ``q[v][e][b*n + a]`` flattened, ``e = j*nx + i``.
"""
from __future__ import annotations

import ctypes
import dataclasses
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "cpr_oracle.c")
_HDR = os.path.join(_HERE, "oracle.h")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

ADVECTION, EULER = 0, 1
GAUSS, LOBATTO = 0, 1
DIV_LP, DIV_CHAIN = 0, 1
RUSANOV, UPWIND, ROE = 0, 1, 2
PERIODIC, TRANSMISSIVE = 0, 1
CPR, FV_MUSCL, FV_MUSCL3 = 0, 1, 2
CORR_GDG, CORR_NDG, CORR_NDG_LUMPED = 0, 1, 2


def build(force: bool = False) -> str:
    """Compile liboracle.so next to its source (OpenMP when available)."""
    newest = max(os.path.getmtime(_SRC), os.path.getmtime(_HDR))
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= newest:
        return _LIB
    base = ["gcc", "-std=c11", "-O2", "-fPIC", "-shared", "-ffp-contract=off",
            "-fno-fast-math", _SRC, "-o", _LIB + ".tmp", "-lm"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True,
                       capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    os.replace(_LIB + ".tmp", _LIB)
    return _LIB


class _Cfg(ctypes.Structure):
    _fields_ = [
        ("eqn", ctypes.c_int), ("nx", ctypes.c_int), ("ny", ctypes.c_int),
        ("p", ctypes.c_int),
        ("x0", ctypes.c_double), ("x1", ctypes.c_double),
        ("y0", ctypes.c_double), ("y1", ctypes.c_double),
        ("pts", ctypes.c_int), ("div", ctypes.c_int), ("flux", ctypes.c_int),
        ("ax", ctypes.c_double), ("ay", ctypes.c_double),
        ("gamma", ctypes.c_double),
        ("bc_x", ctypes.c_int), ("bc_y", ctypes.c_int),
        ("limiter", ctypes.c_int), ("tvb_M", ctypes.c_double),
        ("lim_eps", ctypes.c_double), ("cfl", ctypes.c_double),
        ("scheme", ctypes.c_int), ("corr", ctypes.c_int),
    ]


class _Tab(ctypes.Structure):
    _fields_ = [
        ("n", ctypes.c_int),
        ("xi", ctypes.c_double * 7), ("w", ctypes.c_double * 7),
        ("D", (ctypes.c_double * 7) * 7),
        ("lm", ctypes.c_double * 7), ("lp", ctypes.c_double * 7),
        ("dgl", ctypes.c_double * 7), ("dgr", ctypes.c_double * 7),
    ]


class _Norms(ctypes.Structure):
    _fields_ = [
        ("sum_avg", ctypes.c_double * 4), ("l2_abs", ctypes.c_double),
        ("l2_rel", ctypes.c_double), ("max_wave", ctypes.c_double),
        ("n_nonphys", ctypes.c_longlong),
    ]


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            D, I, L = ctypes.c_double, ctypes.c_int, ctypes.c_long
            P = ctypes.c_void_p
            cp = ctypes.POINTER(_Cfg)
            lib.oracle_legendre.restype = D
            lib.oracle_legendre.argtypes = [I, D]
            lib.oracle_legendre_d.restype = D
            lib.oracle_legendre_d.argtypes = [I, D]
            lib.oracle_tables.restype = I
            lib.oracle_tables.argtypes = [I, I, ctypes.POINTER(_Tab)]
            lib.oracle_tables_corr.restype = I
            lib.oracle_tables_corr.argtypes = [I, I, I, ctypes.POINTER(_Tab)]
            lib.oracle_state_size.restype = L
            lib.oracle_state_size.argtypes = [cp]
            for name in ("oracle_point_coords", "oracle_residual", "oracle_averages",
                         "oracle_residual_jvp", "oracle_residual_vjp"):
                getattr(lib, name).restype = I
            lib.oracle_point_coords.argtypes = [cp, P, P]
            lib.oracle_common_flux.restype = None
            lib.oracle_common_flux.argtypes = [cp, P, P, D, D, P]
            lib.oracle_residual.argtypes = [cp, P, P]
            lib.oracle_averages.argtypes = [cp, P, P]
            lib.oracle_limit.restype = L
            lib.oracle_limit.argtypes = [cp, P, P, P]
            lib.oracle_max_wave.restype = D
            lib.oracle_max_wave.argtypes = [cp, P]
            lib.oracle_dt.restype = D
            lib.oracle_dt.argtypes = [cp, P]
            lib.oracle_rk3_step.restype = I
            lib.oracle_rk3_step.argtypes = [cp, P, D]
            lib.oracle_run.restype = L
            lib.oracle_run.argtypes = [cp, P, L, D, D, ctypes.POINTER(D)]
            lib.oracle_norms.restype = I
            lib.oracle_norms.argtypes = [cp, P, P, ctypes.POINTER(_Norms)]
            lib.oracle_exact_averages.restype = I
            lib.oracle_exact_averages.argtypes = [cp, I, P, D, P]
            lib.oracle_rho_avg_error.restype = D
            lib.oracle_rho_avg_error.argtypes = [cp, P, P]
            lib.oracle_residual_jvp.argtypes = [cp, P, P, P]
            lib.oracle_residual_vjp.argtypes = [cp, P, P, P]
            lib.oracle_rk3_vjp.restype = I
            lib.oracle_rk3_vjp.argtypes = [cp, P, D, P, P]
            lib.oracle_threads.restype = I
            lib.oracle_threads.argtypes = []
            lib.oracle_set_threads.restype = None
            lib.oracle_set_threads.argtypes = [I]
            _lib = lib
    return _lib


@dataclasses.dataclass
class Config:
    """Problem description for the oracle (mirrors ``oracle_cfg``)."""
    eqn: int = EULER
    nx: int = 8
    ny: int = 8
    p: int = 2
    x0: float = 0.0
    x1: float = 1.0
    y0: float = 0.0
    y1: float = 1.0
    pts: int = GAUSS
    div: int = DIV_LP
    flux: int = RUSANOV
    ax: float = 1.0
    ay: float = 1.0
    gamma: float = 1.4
    bc_x: int = PERIODIC
    bc_y: int = PERIODIC
    limiter: int = 0
    tvb_M: float = 0.0
    lim_eps: float = 1e-3
    cfl: float = 0.1
    scheme: int = CPR  # FV_MUSCL / FV_MUSCL3: one average per element, p = 0
    corr: int = CORR_GDG  # CPR edge correction: Radau g_DG, or the NDG lift

    @property
    def nvars(self) -> int:
        return 4 if self.eqn == EULER else 1

    @property
    def n(self) -> int:
        return self.p + 1

    @property
    def ne(self) -> int:
        return self.nx * self.ny

    @property
    def shape(self):
        return (self.nvars, self.ne, self.n * self.n)

    def _c(self) -> _Cfg:
        return _Cfg(**dataclasses.asdict(self))


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def _check(rc, what):
    if rc != 0:
        raise ValueError(f"oracle: {what} rejected its arguments")


def tables(p: int, pts: int = GAUSS, corr: int = CORR_GDG) -> dict:
    t = _Tab()
    _check(_load().oracle_tables_corr(p, pts, corr, ctypes.byref(t)), "tables")
    n = t.n
    return {
        "xi": np.array(t.xi[:n]), "w": np.array(t.w[:n]),
        "D": np.array([[t.D[a][l] for l in range(n)] for a in range(n)]),
        "lm": np.array(t.lm[:n]), "lp": np.array(t.lp[:n]),
        "dgl": np.array(t.dgl[:n]), "dgr": np.array(t.dgr[:n]),
    }


def legendre(k: int, x: float) -> float:
    return _load().oracle_legendre(k, x)


def legendre_d(k: int, x: float) -> float:
    return _load().oracle_legendre_d(k, x)


def point_coords(cfg: Config):
    x = np.empty((cfg.ne, cfg.n * cfg.n))
    y = np.empty_like(x)
    _check(_load().oracle_point_coords(ctypes.byref(cfg._c()), _ptr(x), _ptr(y)), "coords")
    return x, y


def common_flux(cfg: Config, qm, qp, nx: float, ny: float) -> np.ndarray:
    qm, qp = _f64(qm), _f64(qp)
    out = np.empty(cfg.nvars)
    _load().oracle_common_flux(ctypes.byref(cfg._c()), _ptr(qm), _ptr(qp), nx, ny, _ptr(out))
    return out


def residual(cfg: Config, q) -> np.ndarray:
    q = _f64(q).reshape(cfg.shape)
    R = np.empty_like(q)
    _check(_load().oracle_residual(ctypes.byref(cfg._c()), _ptr(q), _ptr(R)), "residual")
    return R


def residual_jvp(cfg: Config, q, dq) -> np.ndarray:
    q, dq = _f64(q).reshape(cfg.shape), _f64(dq).reshape(cfg.shape)
    out = np.empty_like(q)
    _check(_load().oracle_residual_jvp(ctypes.byref(cfg._c()), _ptr(q), _ptr(dq), _ptr(out)),
           "residual_jvp")
    return out


def residual_vjp(cfg: Config, q, rbar) -> np.ndarray:
    q, rbar = _f64(q).reshape(cfg.shape), _f64(rbar).reshape(cfg.shape)
    out = np.empty_like(q)
    _check(_load().oracle_residual_vjp(ctypes.byref(cfg._c()), _ptr(q), _ptr(rbar), _ptr(out)),
           "residual_vjp")
    return out


def rk3_vjp(cfg: Config, q, dt: float, qbar_out) -> np.ndarray:
    q, qb = _f64(q).reshape(cfg.shape), _f64(qbar_out).reshape(cfg.shape)
    out = np.empty_like(q)
    _check(_load().oracle_rk3_vjp(ctypes.byref(cfg._c()), _ptr(q), dt, _ptr(qb), _ptr(out)),
           "rk3_vjp")
    return out


def averages(cfg: Config, q) -> np.ndarray:
    q = _f64(q).reshape(cfg.shape)
    avg = np.empty((cfg.nvars, cfg.ne))
    _check(_load().oracle_averages(ctypes.byref(cfg._c()), _ptr(q), _ptr(avg)), "averages")
    return avg


def limit(cfg: Config, q):
    """Return (limited copy of q, marks[e], margin[e], count)."""
    q = _f64(q).reshape(cfg.shape).copy()
    marks = np.zeros(cfg.ne, dtype=np.int32)
    margin = np.zeros(cfg.ne)
    cnt = _load().oracle_limit(ctypes.byref(cfg._c()), _ptr(q), _ptr(marks), _ptr(margin))
    if cnt < 0:
        raise ValueError("oracle: limit rejected its arguments")
    return q, marks, margin, int(cnt)


def max_wave(cfg: Config, q) -> float:
    q = _f64(q).reshape(cfg.shape)
    return _load().oracle_max_wave(ctypes.byref(cfg._c()), _ptr(q))


def dt(cfg: Config, q) -> float:
    q = _f64(q).reshape(cfg.shape)
    return _load().oracle_dt(ctypes.byref(cfg._c()), _ptr(q))


def rk3_step(cfg: Config, q, dt_: float) -> np.ndarray:
    q = _f64(q).reshape(cfg.shape).copy()
    _check(_load().oracle_rk3_step(ctypes.byref(cfg._c()), _ptr(q), dt_), "rk3_step")
    return q


def run(cfg: Config, q, nsteps: int, dt_: float = 0.0, t_end: float = 0.0, t0: float = 0.0):
    """Return (state, steps taken, final time)."""
    q = _f64(q).reshape(cfg.shape).copy()
    t = ctypes.c_double(t0)
    n = _load().oracle_run(ctypes.byref(cfg._c()), _ptr(q), nsteps, dt_, t_end, ctypes.byref(t))
    if n < 0:
        raise ValueError("oracle: run failed")
    return q, int(n), t.value


def norms(cfg: Config, q, ref=None) -> dict:
    q = _f64(q).reshape(cfg.shape)
    out = _Norms()
    rp = None
    if ref is not None:
        ref = _f64(ref).reshape(cfg.shape)
        rp = _ptr(ref)
    _check(_load().oracle_norms(ctypes.byref(cfg._c()), _ptr(q), rp, ctypes.byref(out)), "norms")
    return {"sum_avg": np.array(out.sum_avg[:cfg.nvars]), "l2_abs": out.l2_abs,
            "l2_rel": out.l2_rel, "max_wave": out.max_wave, "n_nonphys": out.n_nonphys}


def exact_averages(cfg: Config, kind: str, t: float, par=None) -> np.ndarray:
    """kind 'advection' or 'vortex' (par = (eps, xc, yc, uinf, vinf))."""
    k = 0 if kind == "advection" else 1
    V = 1 if k == 0 else 4
    avg = np.empty((V, cfg.ne))
    parr = _f64(par if par is not None else [0.0] * 5)
    _check(_load().oracle_exact_averages(ctypes.byref(cfg._c()), k, _ptr(parr), t, _ptr(avg)),
           "exact_averages")
    return avg


def rho_avg_error(cfg: Config, q, exact_avg) -> float:
    q = _f64(q).reshape(cfg.shape)
    ex = _f64(exact_avg)
    return _load().oracle_rho_avg_error(ctypes.byref(cfg._c()), _ptr(q), _ptr(ex))


def threads() -> int:
    return _load().oracle_threads()


def set_threads(n: int) -> None:
    _load().oracle_set_threads(n)
