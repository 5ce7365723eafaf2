"""GB300-native CPR (Correction Procedure via Reconstruction) hot path.

The kernels live in ``libcpr.so`` (CUDA for sm_103a, C ABI in ``include/cpr.h``);
:mod:`._native` is the ctypes binding and :mod:`.inputs` the seeded synthetic
initial conditions.
"""
from . import adjoint, inputs  # noqa: F401
from ._native import (  # noqa: F401
    ADVECTION, CORR_GDG, Batch, Config, Context, CprError, DIV_CHAIN, DIV_LP, EULER, F32, F64, GAUSS,
    LOBATTO, PERIODIC, RUSANOV, TRANSMISSIVE, UPWIND, load,
)
