"""Seeded synthetic workloads for the CPM Schwarz solver.

This module is shared by the CUDA path's tests/bench and by the CPU oracle. It holds
problem *definitions* only: surface parameters, grid spacings, right-hand-side functions
evaluated at caller-supplied surface points, and seeded random draws (subdomain leaf
weights, trigonometric mode coefficients, serving arrivals). It holds none of the
method's arithmetic (no closest points, no interpolation, no operators, no partitioning).

Workloads (synthetic stand-ins for the paper's sphere / torus / Stanford-Bunny runs):

* ``sphere_small``   unit sphere, h=0.1,   p=3, c=1,  f=(c+12)xyz, 8 RCB subdomains,
                     overlap 2, RAS, FP64, FGMRES(50) to 1e-10.
* ``sphere_h0025``   unit sphere, h=0.025, p=3, c=1,  f=(c+12)xyz, 64 RCB subdomains,
                     overlap 3, ORAS alpha=4 alpha_x=40, FP64 vs FP32 factors, 1e-8.
* ``torus_h00125``   torus R=1 r=0.4, h=0.0125, p=3, c=10, 16 seeded trig modes (std 1),
                     512 subdomains from seeded random-weight RCB, overlap 2, ORAS,
                     BF16-input / FP32-accumulate factors, 1e-8.

u = xyz restricted to the unit sphere is a degree-3 spherical harmonic, so
-Lap_S(xyz) = 3*4*xyz and (c - Lap_S) xyz = (c+12) xyz.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np


@dataclasses.dataclass(frozen=True)
class Workload:
    name: str
    surface: str            # "sphere" | "torus"
    R: float                # sphere radius / torus major radius
    r: float                # torus minor radius (unused for the sphere)
    h: float
    p: int
    c: float
    rhs: str                # "xyz" | "torus_modes"
    n_sub: int
    n_overlap: int
    method: str             # "ras" | "oras"
    alpha: float
    alpha_x: float
    precision: str          # "fp64" | "fp32" | "bf16"
    tol: float
    restart: int = 50
    max_it: int = 500
    weight_seed: int | None = None   # None: equal RCB leaf weights
    rhs_seed: int | None = None


WORKLOADS = {
    "sphere_small": Workload("sphere_small", "sphere", 1.0, 0.0, 0.1, 3, 1.0, "xyz",
                             8, 2, "ras", 0.0, 0.0, "fp64", 1e-10),
    "sphere_h0025": Workload("sphere_h0025", "sphere", 1.0, 0.0, 0.025, 3, 1.0, "xyz",
                             64, 3, "oras", 4.0, 40.0, "fp32", 1e-8),
    "torus_h00125": Workload("torus_h00125", "torus", 1.0, 0.4, 0.0125, 3, 10.0, "torus_modes",
                             512, 2, "oras", 4.0, 40.0, "bf16", 1e-8,
                             weight_seed=3, rhs_seed=33),
    # small case of the same kernels for profiler captures (factors ~1.5 GB, above L2)
    "sphere_h005": Workload("sphere_h005", "sphere", 1.0, 0.0, 0.05, 3, 1.0, "xyz",
                            16, 3, "oras", 4.0, 40.0, "fp32", 1e-8),
}


def leaf_weights(n_sub: int, seed: int | None) -> np.ndarray | None:
    """Integer RCB leaf weights, uniform in [256, 1024] from PCG64(seed); None = equal."""
    if seed is None:
        return None
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.integers(256, 1025, size=n_sub, dtype=np.int64)


def torus_modes(seed: int, n_modes: int = 16):
    """Coefficients of f = sum_k a_k cos(m_k theta + n_k phi + psi_k) drawn from PCG64(seed)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    m = rng.integers(0, 7, size=n_modes)
    n = rng.integers(0, 7, size=n_modes)
    a = rng.standard_normal(n_modes)
    psi = rng.uniform(0.0, 2.0 * math.pi, size=n_modes)
    return m, n, a, psi


def rhs_at_points(wl: Workload, Y: np.ndarray) -> np.ndarray:
    """Right-hand side f evaluated at surface points Y (N x 3), before any normalisation."""
    Y = np.asarray(Y, dtype=np.float64)
    if wl.rhs == "xyz":
        return (wl.c + 12.0) * (Y[:, 0] * Y[:, 1] * Y[:, 2])
    if wl.rhs == "torus_modes":
        m, n, a, psi = torus_modes(wl.rhs_seed)
        theta = np.arctan2(Y[:, 1], Y[:, 0])
        rho = np.sqrt(Y[:, 0] * Y[:, 0] + Y[:, 1] * Y[:, 1])
        phi = np.arctan2(Y[:, 2], rho - wl.R)
        f = np.zeros(len(Y))
        for k in range(len(a)):
            f += a[k] * np.cos(m[k] * theta + n[k] * phi + psi[k])
        return f
    raise ValueError(wl.rhs)


def rhs(wl: Workload, Y: np.ndarray) -> np.ndarray:
    """f at the closest points Y of the active nodes; torus modes are scaled to sample std 1."""
    f = rhs_at_points(wl, Y)
    if wl.rhs == "torus_modes":
        f = f / np.std(f)
    return f


def exact_solution(wl: Workload, Y: np.ndarray) -> np.ndarray | None:
    """Known continuous solution at surface points, where the workload has one."""
    if wl.rhs == "xyz" and wl.surface == "sphere" and wl.R == 1.0:
        return Y[:, 0] * Y[:, 1] * Y[:, 2]
    return None


def random_vector(n: int, seed: int) -> np.ndarray:
    """Seeded standard-normal FP64 vector (operator / preconditioner parity inputs)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.standard_normal(n)


def poisson_arrivals(n_req: int, rate_per_s: float, seed: int = 5) -> np.ndarray:
    """Arrival times (s) of a Poisson request stream."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return np.cumsum(rng.exponential(1.0 / rate_per_s, size=n_req))
