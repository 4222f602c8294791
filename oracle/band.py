"""Computational band: active set Sigma_A, ghost set Sigma_G, canonical order (Sec. 2.1).

Grid nodes are x = (i, j, k) * h with integer (i, j, k), computed as float(i) * h.
Tube-radius construction: Sigma_A = { x : ||x - CP(x)||_2 <= lam }.  Sigma_G = the
6-neighbours of Sigma_A that are not in Sigma_A (nodes completing the 7-point stencils).
Algorithmic construction (the active nodes are the nodes used for interpolation): the
smallest set containing the grid nodes within h of the surface and the interpolation
stencils of CP(x) for its nodes and their 6-neighbours (build_band_algorithmic).

Readings (the paper gives no radius):
  lam = lam_over_h * h with lam_over_h = ((1.0033 * sqrt(3)) * (p + 1)) / 2 by default.
  With p = 2 this is 2.6067 h, inside the interval (2.60641, 2.60699) h that reproduces
  all six unit-sphere active counts the paper prints (Secs. 6.2 and 6.6).
Canonical order: actives lexicographic in (i, j, k), k fastest; ghosts follow, in the same
order. Node index g in [0, N_A) is active, [N_A, N_A + N_G) is a ghost.
Neighbour slots: (-x, +x, -y, +y, -z, +z).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

NBR_OFFSETS = np.array([[-1, 0, 0], [1, 0, 0], [0, -1, 0], [0, 1, 0], [0, 0, -1], [0, 0, 1]],
                       dtype=np.int64)


def default_lam_over_h(p: int) -> float:
    return ((1.0033 * math.sqrt(3.0)) * (p + 1)) / 2.0


@dataclasses.dataclass
class Band:
    surface: object
    h: float
    p: int
    lam: float
    ijk: np.ndarray          # (N_A + N_G, 3) int64, actives then ghosts
    n_active: int
    n_ghost: int
    cp: np.ndarray           # (N_A + N_G, 3) closest points
    grid_lo: np.ndarray      # (3,) lowest (i, j, k) of the index grid
    grid: np.ndarray         # dense int64 index grid, -1 = not a band node
    nbr: np.ndarray          # (N_A, 6) node indices of the 6 neighbours of each active
    tri: np.ndarray | None = None   # triangle holding CP(x) per node (triangulated surfaces)

    @property
    def n_nodes(self) -> int:
        return self.n_active + self.n_ghost

    def lookup(self, IJK: np.ndarray) -> np.ndarray:
        """Node index of grid points IJK (M, 3); -1 where the point is not a band node."""
        rel = IJK - self.grid_lo
        ok = np.all((rel >= 0) & (rel < np.array(self.grid.shape)), axis=1)
        out = np.full(len(IJK), -1, dtype=np.int64)
        r = rel[ok]
        out[ok] = self.grid[r[:, 0], r[:, 1], r[:, 2]]
        return out

    def node_normals(self, idx: np.ndarray) -> np.ndarray:
        """Unit surface normal at CP(x) of the given nodes: analytic for the sphere and the
        torus, the face normal of the triangle holding CP(x) for a triangulated surface."""
        if self.tri is not None:
            return self.surface.normal_of(self.tri[idx])
        return self.surface.normal(self.cp[idx])

    def coords(self, idx=None) -> np.ndarray:
        ijk = self.ijk if idx is None else self.ijk[idx]
        return ijk.astype(np.float64) * self.h


def _grid_range(surface, h: float, lam: float):
    lo, hi = surface.bbox()
    imin = np.floor((lo - lam) / h).astype(np.int64) - 1
    imax = np.ceil((hi + lam) / h).astype(np.int64) + 1
    return imin, imax


def _cp_tri(surface, X: np.ndarray, dmax=None):
    """CP(X) and, for a triangulated surface, the triangle index (else None)."""
    if hasattr(surface, "cp_tri"):
        return surface.cp_tri(X, dmax)
    return surface.cp(X), None


def _tube_test(surface, IJK: np.ndarray, h: float, lam: float):
    X = IJK.astype(np.float64) * h
    Y, tri = _cp_tri(surface, X, lam)
    D = X - Y
    dist = np.sqrt((D[:, 0] * D[:, 0] + D[:, 1] * D[:, 1]) + D[:, 2] * D[:, 2])
    with np.errstate(invalid="ignore"):
        keep = dist <= lam                   # NaN (undefined CP) compares False
    return keep, Y, tri


def _slab_points(i: int, imin, imax):
    J, K = np.meshgrid(np.arange(imin[1], imax[1] + 1), np.arange(imin[2], imax[2] + 1),
                       indexing="ij")
    IJK = np.empty((J.size, 3), dtype=np.int64)
    IJK[:, 0] = i
    IJK[:, 1] = J.ravel()
    IJK[:, 2] = K.ravel()
    return IJK


def active_nodes(surface, h: float, p: int, lam_over_h: float | None = None):
    """Enumerate every grid node of the surface's bounding box (grown by lam) slab by slab
    and keep those within lam of the surface. Returns (ijk, cp, lam) in canonical order."""
    if lam_over_h is None:
        lam_over_h = default_lam_over_h(p)
    lam = lam_over_h * h
    imin, imax = _grid_range(surface, h, lam)
    ijk_parts, cp_parts, tri_parts = [], [], []
    for i in range(int(imin[0]), int(imax[0]) + 1):
        IJK = _slab_points(i, imin, imax)
        keep, Y, tri = _tube_test(surface, IJK, h, lam)
        ijk_parts.append(IJK[keep])
        cp_parts.append(Y[keep])
        if tri is not None:
            tri_parts.append(tri[keep])
    tri = np.concatenate(tri_parts) if tri_parts else None
    return np.concatenate(ijk_parts), np.concatenate(cp_parts), lam, tri


def count_active(surface, h: float, p: int, lam_over_h: float | None = None) -> int:
    """N_A only (for the printed-count pins); same test as active_nodes."""
    return len(active_nodes(surface, h, p, lam_over_h)[0])


def build_band(surface, h: float, p: int, lam_over_h: float | None = None) -> Band:
    """Tube-radius band (Sec. 2.1)."""
    ijk_a, cp_a, lam, tri_a = active_nodes(surface, h, p, lam_over_h)
    return _assemble(surface, h, p, lam, ijk_a, cp_a, tri_a)


def build_band_algorithmic(surface, h: float, p: int) -> Band:
    """Algorithmic band (Sec. 2.1: the active nodes are the nodes used for interpolation).

    Reading: Sigma_A is the smallest node set that contains the seed -- the grid nodes within
    h of the surface, so every surface point has a seed node next to it -- and the
    (p+1)^3 interpolation stencil of CP(x) for every x in Sigma_A and every 6-neighbour x of
    Sigma_A (the ghost nodes need their extension too).  Computed as a closure: process
    the newly added nodes and their 6-neighbours, add their stencils, repeat."""
    seed_ijk, _, _, _ = active_nodes(surface, h, p, 1.0)
    off = np.stack(np.meshgrid(np.arange(p + 1), np.arange(p + 1), np.arange(p + 1), indexing="ij"),
                   axis=-1).reshape(-1, 3)
    members = set(map(tuple, seed_ijk.tolist()))
    processed = set()
    frontier = np.asarray(seed_ijk, dtype=np.int64)
    while len(frontier):
        cand = np.unique(np.concatenate([frontier] + [frontier + o for o in NBR_OFFSETS]), axis=0)
        cand = np.array([q for q in map(tuple, cand.tolist()) if q not in processed], dtype=np.int64)
        if len(cand) == 0:
            break
        processed.update(map(tuple, cand.tolist()))
        Y, _ = _cp_tri(surface, cand.astype(np.float64) * h)
        if np.any(~np.isfinite(Y)):
            raise ValueError("algorithmic band reaches a point without a closest point")
        base = np.floor(Y / h - (p - 1) / 2.0).astype(np.int64)
        sten = np.unique((base[:, None, :] + off[None, :, :]).reshape(-1, 3), axis=0)
        new = [q for q in map(tuple, sten.tolist()) if q not in members]
        members.update(new)
        frontier = np.array(new, dtype=np.int64).reshape(-1, 3)
    ijk_a = np.array(sorted(members), dtype=np.int64)          # lexicographic, k fastest
    cp_a, tri_a = _cp_tri(surface, ijk_a.astype(np.float64) * h)
    return _assemble(surface, h, p, 0.0, ijk_a, cp_a, tri_a)


def _assemble(surface, h, p, lam, ijk_a, cp_a, tri_a) -> Band:
    """Grid, ghosts, neighbour table of a band given its actives in canonical order."""
    n_a = len(ijk_a)
    lo = ijk_a.min(0) - 2
    hi = ijk_a.max(0) + 2
    shape = tuple((hi - lo + 1).tolist())
    grid = np.full(shape, -1, dtype=np.int64)
    ra = ijk_a - lo
    grid[ra[:, 0], ra[:, 1], ra[:, 2]] = np.arange(n_a)
    # ghosts: 6-neighbours of actives that are not active, in lexicographic order
    cand = (ijk_a[:, None, :] + NBR_OFFSETS[None, :, :]).reshape(-1, 3)
    rc = cand - lo
    is_new = grid[rc[:, 0], rc[:, 1], rc[:, 2]] < 0
    ghosts = np.unique(cand[is_new], axis=0)            # lexicographic (i, j, k)
    n_g = len(ghosts)
    rg = ghosts - lo
    grid[rg[:, 0], rg[:, 1], rg[:, 2]] = n_a + np.arange(n_g)
    cp_g, tri_g = _cp_tri(surface, ghosts.astype(np.float64) * h)
    ijk = np.concatenate([ijk_a, ghosts])
    cp = np.concatenate([cp_a, cp_g])
    tri = None if tri_a is None else np.concatenate([tri_a, tri_g])
    nb = (ijk_a[:, None, :] + NBR_OFFSETS[None, :, :]) - lo
    nbr = grid[nb[..., 0], nb[..., 1], nb[..., 2]]
    assert np.all(nbr >= 0)
    return Band(surface, h, p, lam, ijk, n_a, n_g, cp, lo, grid, nbr, tri)
