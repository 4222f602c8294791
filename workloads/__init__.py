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
* ``mesh_h001``      perturbed icosphere (icosahedron subdivided 6 times, 81,920 triangles,
                     vertex radius 1 + 0.15 g(v)/max|g| with 8 seeded ambient modes g, seed 4),
                     h=0.01, p=3, c=1, f = 8 seeded ambient modes (seed 44, std 1),
                     256 RCB subdomains, overlap 3, ORAS, FP32 factors, 1e-8.
                     Stands in for the paper's Stanford-Bunny runs (a triangulated surface).

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
    mesh_level: int = 0              # triangulated surfaces: icosphere subdivisions
    mesh_amp: float = 0.0            #   relative radial perturbation amplitude
    mesh_seed: int | None = None     #   seed of the perturbation modes


WORKLOADS = {
    "sphere_small": Workload("sphere_small", "sphere", 1.0, 0.0, 0.1, 3, 1.0, "xyz",
                             8, 2, "ras", 0.0, 0.0, "fp64", 1e-10),
    "sphere_h0025": Workload("sphere_h0025", "sphere", 1.0, 0.0, 0.025, 3, 1.0, "xyz",
                             64, 3, "oras", 4.0, 40.0, "fp32", 1e-8),
    "torus_h00125": Workload("torus_h00125", "torus", 1.0, 0.4, 0.0125, 3, 10.0, "torus_modes",
                             512, 2, "oras", 4.0, 40.0, "bf16", 1e-8,
                             weight_seed=3, rhs_seed=33),
    "mesh_h001": Workload("mesh_h001", "trimesh", 1.0, 0.0, 0.01, 3, 1.0, "ambient_modes",
                          256, 3, "oras", 4.0, 40.0, "fp32", 1e-8, rhs_seed=44,
                          mesh_level=6, mesh_amp=0.15, mesh_seed=4),
    # small triangulated case (1,280 triangles) for oracle / parity tests
    "mesh_small": Workload("mesh_small", "trimesh", 1.0, 0.0, 0.05, 3, 1.0, "ambient_modes",
                           8, 2, "oras", 4.0, 40.0, "fp64", 1e-10, rhs_seed=44,
                           mesh_level=3, mesh_amp=0.15, mesh_seed=4),
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


def ambient_modes(seed: int, n_modes: int = 8):
    """g(x) = sum_k b_k cos(w_k . x + psi_k): b_k ~ N(0,1), w_k uniform direction with
    |w_k| uniform in [1, 3], psi_k uniform in [0, 2 pi), all from PCG64(seed)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    b = rng.standard_normal(n_modes)
    d = rng.standard_normal((n_modes, 3))
    d /= np.linalg.norm(d, axis=1)[:, None]
    w = d * rng.uniform(1.0, 3.0, size=n_modes)[:, None]
    psi = rng.uniform(0.0, 2.0 * math.pi, size=n_modes)
    return b, w, psi


def eval_ambient_modes(modes, X: np.ndarray) -> np.ndarray:
    b, w, psi = modes
    return np.cos(np.asarray(X, dtype=np.float64) @ w.T + psi[None, :]) @ b


def icosphere(level: int):
    """Unit icosphere: the regular icosahedron (vertices (0, +-1, +-phi) and cyclic
    permutations, projected to the unit sphere) with every triangle split into four
    `level` times, new vertices projected to the sphere.  Triangles wound outward."""
    phi = (1.0 + math.sqrt(5.0)) / 2.0
    V = []
    for a in (-1.0, 1.0):
        for b in (-phi, phi):
            V += [(0.0, a, b), (a, b, 0.0), (b, 0.0, a)]
    V = np.array(V)
    # faces: vertex triples that are pairwise at edge length 2
    D = np.linalg.norm(V[:, None, :] - V[None, :, :], axis=2)
    adj = np.abs(D - 2.0) < 1e-9
    T = [(i, j, k) for i in range(12) for j in range(i + 1, 12) for k in range(j + 1, 12)
         if adj[i, j] and adj[j, k] and adj[i, k]]
    V = V / np.linalg.norm(V, axis=1)[:, None]
    T = np.array(T, dtype=np.int64)
    for _ in range(level):
        verts = [tuple(v) for v in V]
        mid = {}

        def midpoint(i, j):
            key = (min(i, j), max(i, j))
            if key not in mid:
                m = (np.asarray(verts[i]) + np.asarray(verts[j])) / 2.0
                verts.append(tuple(m / np.linalg.norm(m)))
                mid[key] = len(verts) - 1
            return mid[key]

        newT = []
        for a, b, c in T:
            ab, bc, ca = midpoint(a, b), midpoint(b, c), midpoint(c, a)
            newT += [(a, ab, ca), (ab, b, bc), (ca, bc, c), (ab, bc, ca)]
        V = np.array(verts)
        T = np.array(newT, dtype=np.int64)
    # outward winding: (b - a) x (c - a) points away from the origin
    A, B, C = V[T[:, 0]], V[T[:, 1]], V[T[:, 2]]
    flip = np.einsum("ij,ij->i", np.cross(B - A, C - A), A + B + C) < 0
    T[flip] = T[flip][:, [0, 2, 1]]
    return V, T.astype(np.int32)


def perturbed_icosphere(level: int, amp: float, seed: int):
    """Icosphere with vertex radius 1 + amp g(v)/max_v |g(v)| (g: 8 ambient modes)."""
    V, T = icosphere(level)
    g = eval_ambient_modes(ambient_modes(seed), V)
    rad = 1.0 + amp * g / np.max(np.abs(g))
    return V * rad[:, None], T


_MESH_CACHE = {}


def surface_mesh(wl: Workload):
    """(verts, tris) of a triangulated workload, None for analytic surfaces."""
    if wl.surface != "trimesh":
        return None
    key = (wl.mesh_level, wl.mesh_amp, wl.mesh_seed)
    if key not in _MESH_CACHE:
        _MESH_CACHE[key] = perturbed_icosphere(wl.mesh_level, wl.mesh_amp, wl.mesh_seed)
    return _MESH_CACHE[key]


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
    if wl.rhs == "ambient_modes":
        return eval_ambient_modes(ambient_modes(wl.rhs_seed), Y)
    raise ValueError(wl.rhs)


def rhs(wl: Workload, Y: np.ndarray) -> np.ndarray:
    """f at the closest points Y of the active nodes; torus modes are scaled to sample std 1."""
    f = rhs_at_points(wl, Y)
    if wl.rhs in ("torus_modes", "ambient_modes"):
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


# ---------------------------------------------------------------- serving stream
SERVING_SURFACES = ("sphere", "torus", "mesh")
SERVING_H = (0.05, 0.025, 0.0125)
SERVING_H_PROB = (0.5, 0.35, 0.15)


@dataclasses.dataclass(frozen=True)
class ServingRequestSpec:
    """One request of the serving stream: operator (surface, h, c), right-hand sides and an
    optional backward-Euler chain (c = 1/dt, rhs_{n+1} = u_n / dt, same factorisation)."""
    rid: int
    surface: str            # "sphere" | "torus" | "mesh" (the 81,920-triangle workload mesh)
    h: float
    c: float
    nrhs: int
    rhs_seed: int
    chain_steps: int        # backward-Euler steps after the first solve (0: plain solve)


def serving_stream(n_req: int, seed: int = 5, repeat_prob: float = 0.3, chain_prob: float = 0.25,
                   max_nrhs: int = 32, h_choices=SERVING_H, h_prob=SERVING_H_PROB):
    """Seeded request mix: surface uniform over sphere / torus(1, 0.4) / perturbed-icosphere
    mesh, h from h_choices with probabilities h_prob, c log-uniform in [0.1, 100], 1..max_nrhs
    smooth right-hand sides (log-uniform), a fraction of backward-Euler chains (2-6 steps, one
    rhs) and a fraction of requests that reuse an earlier request's operator (same surface, h
    and c), which is what lets factorisations and batches be shared."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for i in range(n_req):
        if out and rng.uniform() < repeat_prob:
            prev = out[int(rng.integers(0, len(out)))]
            surface, h, c = prev.surface, prev.h, prev.c
        else:
            surface = SERVING_SURFACES[int(rng.integers(0, len(SERVING_SURFACES)))]
            h = float(h_choices[int(rng.choice(len(h_choices), p=np.asarray(h_prob) / np.sum(h_prob)))])
            c = float(10.0 ** rng.uniform(-1.0, 2.0))
        if rng.uniform() < chain_prob:
            nrhs, steps = 1, int(rng.integers(2, 7))
        else:
            nrhs = int(min(max_nrhs, np.floor(np.exp(rng.uniform(0.0, math.log(max_nrhs + 1))))))
            nrhs, steps = max(1, nrhs), 0
        out.append(ServingRequestSpec(i, surface, h, c, nrhs, int(rng.integers(0, 2 ** 31)), steps))
    return out


def smooth_rhs(Y: np.ndarray, seed: int, nrhs: int) -> np.ndarray:
    """nrhs smooth right-hand sides (8 ambient modes each, std 1) at surface points Y."""
    F = np.empty((nrhs, len(Y)))
    for k in range(nrhs):
        f = eval_ambient_modes(ambient_modes(seed + 7919 * k), Y)
        F[k] = f / np.std(f)
    return F
