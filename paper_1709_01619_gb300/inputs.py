"""Seeded synthetic inputs for the CPR solver: initial conditions and noise.

This module holds only problem definitions (initial states evaluated at given
point coordinates) and seeded random numbers.  It contains none of the
method's arithmetic, so both the CUDA path and its test oracle may use it.

Coordinates come in as arrays ``x, y`` of shape ``(ne, n*n)`` (one row per
element, points in ``b*n + a`` order); states come out as ``(V, ne, n*n)``
float64 arrays, ``V = 1`` for advection and ``V = 4`` for Euler with
conserved variables ``(rho, rho u, rho v, e)`` (Sec. 2, Eq. 3).
"""
from __future__ import annotations

import math

import numpy as np

GAMMA = 1.4


def conserved(rho, u, v, p, gamma: float = GAMMA) -> np.ndarray:
    """Primitive -> conserved, e = p/(gamma-1) + rho (u^2 + v^2)/2 (Eq. 5)."""
    rho, u, v, p = (np.asarray(a, dtype=np.float64) for a in (rho, u, v, p))
    return np.stack([rho, rho * u, rho * v,
                     p / (gamma - 1.0) + 0.5 * rho * (u * u + v * v)])


def advection_sine(x, y) -> np.ndarray:
    """u0 = sin(2 pi x) sin(2 pi y) on the unit square."""
    return (np.sin(2 * np.pi * x) * np.sin(2 * np.pi * y))[None]


def vortex(x, y, eps: float = 5.0, xc: float = 5.0, yc: float = 5.0,
           uinf: float = 1.0, vinf: float = 1.0, lx: float = 10.0, ly: float = 10.0,
           gamma: float = GAMMA) -> np.ndarray:
    """Isentropic vortex of Sec. 4.1 with mean (rho, u, v, p) = (1, uinf, vinf, 1).

    (du, dv) = eps/(2 pi) exp((1 - r^2)/2) (-ybar, xbar),
    dT = -(gamma-1) eps^2/(8 gamma pi^2) exp(1 - r^2), entropy unchanged.
    Offsets are taken to the nearest periodic image of the centre.
    """
    xb = x - xc
    yb = y - yc
    xb = xb - lx * np.floor(xb / lx + 0.5)
    yb = yb - ly * np.floor(yb / ly + 0.5)
    r2 = xb * xb + yb * yb
    amp = eps / (2 * math.pi) * np.exp(0.5 * (1.0 - r2))
    T = 1.0 - (gamma - 1.0) * eps * eps / (8.0 * gamma * math.pi ** 2) * np.exp(1.0 - r2)
    rho = T ** (1.0 / (gamma - 1.0))
    return conserved(rho, uinf - amp * yb, vinf + amp * xb, rho * T, gamma)


# Four-quadrant Riemann problem on [0,1]^2 split at (0.8, 0.8):
# (rho, u, v, p) per quadrant.  Points exactly on a split line go to the
# upper / right state.
FOUR_QUADRANT = {
    "UR": (1.5, 0.0, 0.0, 1.5),
    "UL": (0.5323, 1.206, 0.0, 0.3),
    "LL": (0.138, 1.206, 1.206, 0.029),
    "LR": (0.5323, 0.0, 1.206, 0.3),
}


def four_quadrant(x, y, split: float = 0.8, gamma: float = GAMMA) -> np.ndarray:
    right = x >= split
    up = y >= split
    prim = np.zeros((4,) + np.shape(x))
    for key, mask in (("UR", right & up), ("UL", ~right & up),
                      ("LL", ~right & ~up), ("LR", right & ~up)):
        for k in range(4):
            prim[k][mask] = FOUR_QUADRANT[key][k]
    return conserved(prim[0], prim[1], prim[2], prim[3], gamma)


def radial_shock(x, y, radius: float = 0.4, gamma: float = GAMMA) -> np.ndarray:
    """Radially expanding shock tube of Sec. 4.2 on [-1,1]^2: (rho, p) = (1, 1)
    inside r < 0.4, (0.125, 0.1) outside, at rest."""
    inside = x * x + y * y < radius * radius
    rho = np.where(inside, 1.0, 0.125)
    p = np.where(inside, 1.0, 0.1)
    z = np.zeros_like(rho)
    return conserved(rho, z, z, p, gamma)


def entropy_wave(x, y, lx: float, ly: float, amp: float = 0.2, u: float = 1.0, v: float = 0.5,
                 p: float = 1.0, gamma: float = GAMMA) -> np.ndarray:
    """Density wave rho = 1 + amp sin(2 pi x / lx) sin(2 pi y / ly) carried by a
    uniform flow (u, v) at uniform pressure: a smooth periodic Euler solution
    on [0, lx] x [0, ly] that is advected unchanged."""
    rho = 1.0 + amp * np.sin(2 * np.pi * x / lx) * np.sin(2 * np.pi * y / ly)
    return conserved(rho, np.full_like(rho, u), np.full_like(rho, v), np.full_like(rho, p), gamma)


def freestream(x, rho=1.0, u=0.7, v=-0.3, p=0.9, gamma: float = GAMMA) -> np.ndarray:
    one = np.ones_like(x)
    return conserved(rho * one, u * one, v * one, p * one, gamma)


def noise(shape, seed: int, scale: float) -> np.ndarray:
    """Uniform noise in [-scale, scale) from numpy's PCG64 stream ``seed``."""
    return scale * (2.0 * np.random.default_rng(seed).random(shape) - 1.0)


def perturbed(q: np.ndarray, seed: int, rel: float = 1e-2) -> np.ndarray:
    """q * (1 + noise): a smooth state made rough at every point, so that every
    table entry and every face takes part in a parity comparison."""
    return q * (1.0 + noise(q.shape, seed, rel))


# CFL number per order for the batch of vortices (Eq. 36 takes the speed
# |V| + c).  The linear stability bound of three-stage SSP Runge-Kutta with
# this scheme in 1D is about 0.21, 0.13 and 0.09 for p = 2, 3, 4 (|a| dt / h);
# in 2D the step must also cover (|u| + c) / hx + (|v| + c) / hy, which for a
# flow along the diagonal of a weak vortex is about 0.6 times the 1D bound in
# these units.  These values keep a margin of about 25-30 % below that.
BATCH_CFL = {2: 0.1, 3: 0.06, 4: 0.04}


def batch_instances(count: int = 64, seed: int = 0):
    """Ragged batch of vortex solves: per instance N ~ U{32..256} elements per
    side, p ~ U{2,3,4}, strength eps ~ U[1,5], all drawn from one seed."""
    rng = np.random.default_rng(seed)
    n = rng.integers(32, 257, size=count)
    p = rng.integers(2, 5, size=count)
    eps = rng.uniform(1.0, 5.0, size=count)
    return [{"N": int(n[k]), "p": int(p[k]), "eps": float(eps[k])} for k in range(count)]
