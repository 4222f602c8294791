"""One-call oracle setup of a workload: band, E, A, partition, local problems, Schwarz.

The steps follow the paper's phases (Sec. 6.6): global meshing (band + partition), global
matrix (E and A), local operators (assembly + LU), then the preconditioned GMRES solve.
"""
from __future__ import annotations

import dataclasses

import numpy as np

from . import band as band_mod
from . import geometry, interp, krylov, local, operator, partition, schwarz


@dataclasses.dataclass
class OracleProblem:
    band: object
    E: object
    A: object
    labels: np.ndarray
    subs: list
    lps: list
    M: schwarz.Schwarz
    c: float
    f: np.ndarray | None = None


def setup(surface_kind: str, R: float, r: float, h: float, p: int, c: float, n_sub: int,
          n_overlap: int, method: str, alpha: float = 4.0, alpha_x: float = 40.0,
          leaf_weights=None, lam_over_h=None, reading: str = "R1",
          dense: bool = False, verts=None, tris=None, align_passes: int = 0,
          split: str = "coordinate") -> OracleProblem:
    surf = geometry.make_surface(surface_kind, R, r, verts, tris)
    B = band_mod.build_band(surf, h, p, lam_over_h)
    E = interp.extension_matrix(B)
    A = operator.cpm_matrix(B, E, c)
    labels = partition.rcb(B.cp[:B.n_active], n_sub, leaf_weights) if split == "coordinate" else \
        partition.graph_bisection(B, n_sub, leaf_weights)
    if align_passes:
        labels = partition.align_interfaces(B, labels, align_passes)
    robin = method == "oras" and reading == "R1"
    subs = partition.all_subdomains(B, E, labels, n_sub, n_overlap, robin)
    if method == "ras":
        lps = [local.ras_local(A, s) for s in subs]
    elif method == "oras":
        cross = partition.cross_point_nodes(B, labels)
        marks = partition.CrossMarks(B, cross, n_overlap)
        lps = [local.oras_local(B, s, c, alpha, alpha_x, marks, reading) for s in subs]
    else:
        raise ValueError(method)
    M = schwarz.Schwarz(lps, B.n_active, dense=dense)
    return OracleProblem(B, E, A, labels, subs, lps, M, c)


def setup_workload(wl, **kw) -> OracleProblem:
    from workloads import leaf_weights, rhs, surface_mesh
    mesh = surface_mesh(wl)
    if mesh is not None:
        kw.setdefault("verts", mesh[0])
        kw.setdefault("tris", mesh[1])
    prob = setup(wl.surface, wl.R, wl.r, wl.h, wl.p, wl.c, wl.n_sub, wl.n_overlap, wl.method,
                 wl.alpha, wl.alpha_x, leaf_weights(wl.n_sub, wl.weight_seed), **kw)
    prob.f = rhs(wl, prob.band.cp[:prob.band.n_active])
    return prob


def solve(prob: OracleProblem, f: np.ndarray, tol: float, restart: int = 50, max_it: int = 1000,
          **kw):
    return krylov.fgmres(lambda x: prob.A @ x, prob.M.apply, f, tol, restart, max_it, **kw)
