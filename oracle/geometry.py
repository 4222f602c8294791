"""Closest-point functions CP_S and surface normals (Sec. 2.1, definition of CP_S).

CP_S(x) = argmin_{y in S} ||x - y||_2.  For the sphere and the torus it has a closed form;
for a triangulated surface it is the closest point over all triangles (exact point-triangle
closest point by Voronoi-region tests, Ericson, Real-Time Collision Detection, Sec. 5.1.5),
ties going to the lowest triangle index.
All arithmetic is FP64 in a fixed operation order (norms as sqrt((x*x + y*y) + z*z), dot
products as (u0 v0 + u1 v1) + u2 v2).
"""
from __future__ import annotations

import numpy as np
from scipy.spatial import cKDTree


def norm3(V: np.ndarray) -> np.ndarray:
    """Euclidean norm of rows of an (N, 3) array, summed x, then y, then z."""
    return np.sqrt((V[:, 0] * V[:, 0] + V[:, 1] * V[:, 1]) + V[:, 2] * V[:, 2])


class Sphere:
    """Sphere of radius R centred at the origin: CP(x) = R x/|x|."""

    kind = "sphere"

    def __init__(self, R: float = 1.0):
        self.R = float(R)

    def bbox(self):
        R = self.R
        return np.array([-R, -R, -R]), np.array([R, R, R])

    def cp(self, X: np.ndarray) -> np.ndarray:
        X = np.asarray(X, dtype=np.float64)
        r = norm3(X)
        with np.errstate(divide="ignore", invalid="ignore"):
            Y = (X / r[:, None]) * self.R
        Y[r == 0.0] = np.nan          # CP undefined at the centre: never in the band
        return Y

    def normal(self, Y: np.ndarray) -> np.ndarray:
        """Unit outward normal at surface points Y."""
        return Y / norm3(Y)[:, None]

    def radial_bounds(self):
        """The set of x with ||x - CP(x)|| <= d is the shell | |x| - R | <= d."""
        return self.R


class Torus:
    """Torus about the z axis with major radius R and minor radius r.

    The ring circle is C(x) = R (x, y, 0)/rho with rho = sqrt(x^2 + y^2); then
    CP(x) = C + r (x - C)/|x - C|.
    """

    kind = "torus"

    def __init__(self, R: float = 1.0, r: float = 0.4):
        self.R = float(R)
        self.r = float(r)

    def bbox(self):
        a = self.R + self.r
        return np.array([-a, -a, -self.r]), np.array([a, a, self.r])

    def _ring(self, X: np.ndarray) -> np.ndarray:
        rho = np.sqrt(X[:, 0] * X[:, 0] + X[:, 1] * X[:, 1])
        C = np.zeros_like(X)
        with np.errstate(divide="ignore", invalid="ignore"):
            C[:, 0] = (X[:, 0] / rho) * self.R
            C[:, 1] = (X[:, 1] / rho) * self.R
        C[rho == 0.0] = np.nan        # CP undefined on the axis: never in the band
        return C

    def cp(self, X: np.ndarray) -> np.ndarray:
        X = np.asarray(X, dtype=np.float64)
        C = self._ring(X)
        V = X - C
        s = norm3(V)
        with np.errstate(divide="ignore", invalid="ignore"):
            Y = C + (V / s[:, None]) * self.r
        Y[s == 0.0] = np.nan          # CP undefined on the ring circle itself
        return Y

    def normal(self, Y: np.ndarray) -> np.ndarray:
        C = self._ring(Y)
        V = Y - C
        return V / norm3(V)[:, None]


def dot3(U: np.ndarray, V: np.ndarray) -> np.ndarray:
    return (U[:, 0] * V[:, 0] + U[:, 1] * V[:, 1]) + U[:, 2] * V[:, 2]


def closest_point_on_triangles(P, A, B, C):
    """Closest point of triangle (A_k, B_k, C_k) to P_k for paired rows (K, 3).

    The plane of the triangle is split into the Voronoi regions of its three vertices, its
    three edges and its face; the first region (in the order a, b, ab, c, ac, bc, face)
    whose dot-product test holds gives the point:
      vertex a   : (b-a).(p-a) <= 0 and (c-a).(p-a) <= 0
      vertex b   : (b-a).(p-b) >= 0 and (c-a).(p-b) <= (b-a).(p-b)
      edge ab    : vc <= 0 with p projecting inside ab       -> a + t (b-a)
      vertex c   : (c-a).(p-c) >= 0 and (b-a).(p-c) <= (c-a).(p-c)
      edge ac    : vb <= 0 with p projecting inside ac       -> a + t (c-a)
      edge bc    : va <= 0 with p projecting inside bc       -> b + t (c-b)
      face       : barycentric (va, vb, vc) / (va + vb + vc)
    where va, vb, vc are the scaled barycentric coordinates of the projection of p.
    """
    AB = B - A
    AC = C - A
    AP = P - A
    d1 = dot3(AB, AP)
    d2 = dot3(AC, AP)
    BP = P - B
    d3 = dot3(AB, BP)
    d4 = dot3(AC, BP)
    vc = d1 * d4 - d3 * d2
    CP = P - C
    d5 = dot3(AB, CP)
    d6 = dot3(AC, CP)
    vb = d5 * d2 - d1 * d6
    va = d3 * d6 - d5 * d4
    left = np.ones(len(P), dtype=bool)            # no region chosen yet

    def take(cond):
        nonlocal left
        m = left & cond
        left = left & ~m
        return m

    m_a = take((d1 <= 0.0) & (d2 <= 0.0))
    m_b = take((d3 >= 0.0) & (d4 <= d3))
    m_ab = take((vc <= 0.0) & (d1 >= 0.0) & (d3 <= 0.0))
    m_c = take((d6 >= 0.0) & (d5 <= d6))
    m_ac = take((vb <= 0.0) & (d2 >= 0.0) & (d6 <= 0.0))
    m_bc = take((va <= 0.0) & ((d4 - d3) >= 0.0) & ((d5 - d6) >= 0.0))
    m_f = left
    Y = np.empty_like(P)
    with np.errstate(divide="ignore", invalid="ignore"):
        Y[m_a] = A[m_a]
        Y[m_b] = B[m_b]
        t = d1[m_ab] / (d1[m_ab] - d3[m_ab])
        Y[m_ab] = A[m_ab] + AB[m_ab] * t[:, None]
        Y[m_c] = C[m_c]
        t = d2[m_ac] / (d2[m_ac] - d6[m_ac])
        Y[m_ac] = A[m_ac] + AC[m_ac] * t[:, None]
        e = d4[m_bc] - d3[m_bc]
        t = e / (e + (d5[m_bc] - d6[m_bc]))
        Y[m_bc] = B[m_bc] + (C[m_bc] - B[m_bc]) * t[:, None]
        den = (va[m_f] + vb[m_f]) + vc[m_f]
        v = vb[m_f] / den
        w = vc[m_f] / den
        Y[m_f] = (A[m_f] + AB[m_f] * v[:, None]) + AC[m_f] * w[:, None]
    return Y


class TriMesh:
    """Triangulated closed surface: vertices (n_v, 3), triangles (n_t, 3) vertex indices.

    CP(x) is the closest point over all triangles (ties: lowest triangle index); the normal
    at a closest point is the unit face normal (b - a) x (c - a) / |(b - a) x (c - a)| of the
    triangle it lies on.  Candidate triangles of a point x come from a k-d tree over the
    triangle centroids: with u = the distance from x to its nearest vertex (>= the distance
    to the surface), the closest triangle has its centroid within u + rho_max of x, where
    rho_max is the largest centroid-to-vertex distance.  That candidate set is a superset
    of the minimisers, so the result is the exact argmin.
    """

    kind = "trimesh"

    def __init__(self, verts, tris):
        self.V = np.ascontiguousarray(verts, dtype=np.float64)
        self.T = np.ascontiguousarray(tris, dtype=np.int64)
        if self.V.ndim != 2 or self.V.shape[1] != 3 or self.T.ndim != 2 or self.T.shape[1] != 3:
            raise ValueError("TriMesh: verts (n,3) and tris (m,3) expected")
        self.A = self.V[self.T[:, 0]]
        self.B = self.V[self.T[:, 1]]
        self.C = self.V[self.T[:, 2]]
        AB = self.B - self.A
        AC = self.C - self.A
        Nrm = np.stack([AB[:, 1] * AC[:, 2] - AB[:, 2] * AC[:, 1],
                        AB[:, 2] * AC[:, 0] - AB[:, 0] * AC[:, 2],
                        AB[:, 0] * AC[:, 1] - AB[:, 1] * AC[:, 0]], axis=1)
        self.face_normal = Nrm / norm3(Nrm)[:, None]
        ctr = (self.A + self.B + self.C) / 3.0
        self.rho_max = float(max(norm3(self.A - ctr).max(), norm3(self.B - ctr).max(),
                                 norm3(self.C - ctr).max()))
        self._ctree = cKDTree(ctr)
        self._vtree = cKDTree(self.V)

    def bbox(self):
        return self.V.min(0), self.V.max(0)

    def cp_tri(self, X: np.ndarray, dmax: float | None = None):
        """(CP(X), triangle index).  With dmax, points farther than dmax from every
        triangle get NaN and index -1 (they are outside any band of radius dmax)."""
        X = np.asarray(X, dtype=np.float64)
        n = len(X)
        Y = np.full((n, 3), np.nan)
        tri = np.full(n, -1, dtype=np.int64)
        for s0 in range(0, n, 65536):
            Xc = X[s0:s0 + 65536]
            ub, _ = self._vtree.query(Xc)
            lim = ub if dmax is None else np.minimum(ub, dmax)
            rad = lim * (1.0 + 1e-9) + 1e-12 + self.rho_max
            lists = self._ctree.query_ball_point(Xc, rad)
            cnt = np.fromiter((len(c) for c in lists), dtype=np.int64, count=len(lists))
            if cnt.sum() == 0:
                continue
            pt = np.repeat(np.arange(len(Xc)), cnt)
            tt = np.fromiter((t for c in lists for t in c), dtype=np.int64, count=int(cnt.sum()))
            Q = Xc[pt]
            Yc = closest_point_on_triangles(Q, self.A[tt], self.B[tt], self.C[tt])
            D = Q - Yc
            d2 = (D[:, 0] * D[:, 0] + D[:, 1] * D[:, 1]) + D[:, 2] * D[:, 2]
            order = np.lexsort((tt, d2, pt))          # by point, then distance, then triangle
            first = order[np.r_[True, pt[order][1:] != pt[order][:-1]]]
            keep = np.ones(len(first), dtype=bool)
            if dmax is not None:
                keep = np.sqrt(d2[first]) <= dmax * (1.0 + 1e-9) + 1e-12
            first = first[keep]
            Y[s0 + pt[first]] = Yc[first]
            tri[s0 + pt[first]] = tt[first]
        return Y, tri

    def cp(self, X: np.ndarray, dmax: float | None = None) -> np.ndarray:
        return self.cp_tri(X, dmax)[0]

    def normal_of(self, tri: np.ndarray) -> np.ndarray:
        return self.face_normal[tri]


def make_surface(kind: str, R: float = 1.0, r: float = 0.0, verts=None, tris=None):
    if kind == "sphere":
        return Sphere(R)
    if kind == "torus":
        return Torus(R, r)
    if kind == "trimesh":
        return TriMesh(verts, tris)
    raise ValueError(kind)
