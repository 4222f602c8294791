"""Pins for the oracle's triangulated-surface closest point (CPU only).

The point-triangle closest point is checked against closed forms (a point in the face, a
point above the face, vertex and edge regions by clamped projections), against a dense
sampling of the triangle, and TriMesh.cp (k-d tree candidates) against a brute-force scan of
every triangle.  The icosphere is checked against the analytic sphere it approximates, and
the perturbed workload surface against the band-width condition lambda < 1/kappa_max.
"""
import math

import numpy as np
import pytest

from oracle import band, geometry, problems, schwarz
from oracle.geometry import closest_point_on_triangles
from workloads import WORKLOADS, icosphere, perturbed_icosphere, surface_mesh

TRI = np.array([[0.1, -0.2, 0.3], [1.3, 0.1, 0.2], [0.4, 0.9, -0.1]])


def _cp(p):
    P = np.atleast_2d(np.asarray(p, dtype=float))
    A, B, C = (np.repeat(TRI[i][None], len(P), 0) for i in range(3))
    return closest_point_on_triangles(P, A, B, C)


def _normal():
    n = np.cross(TRI[1] - TRI[0], TRI[2] - TRI[0])
    return n / np.linalg.norm(n)


def test_point_in_face_is_its_own_closest_point():
    rng = np.random.default_rng(1)
    for _ in range(200):
        w = rng.dirichlet([1, 1, 1])
        x = w @ TRI
        assert np.allclose(_cp(x)[0], x, atol=1e-14)


def test_point_above_face_projects_to_foot():
    rng = np.random.default_rng(2)
    n = _normal()
    for _ in range(200):
        w = rng.dirichlet([2, 2, 2])
        foot = w @ TRI
        x = foot + rng.uniform(-2, 2) * n
        assert np.allclose(_cp(x)[0], foot, atol=1e-13)


def _seg(x, a, b):
    t = np.clip(np.dot(x - a, b - a) / np.dot(b - a, b - a), 0.0, 1.0)
    return a + t * (b - a)


def test_outside_points_match_nearest_edge_or_vertex():
    """A point whose in-plane projection lies outside the triangle has its closest point
    on the boundary: the nearest of the three clamped edge projections."""
    rng = np.random.default_rng(3)
    n = _normal()
    ctr = TRI.mean(0)
    checked = 0
    for _ in range(2000):
        x = ctr + rng.normal(size=3) * 1.5
        y = x - np.dot(x - TRI[0], n) * n                      # in-plane projection
        M = np.column_stack([TRI[1] - TRI[0], TRI[2] - TRI[0], n])
        l1, l2, _ = np.linalg.solve(M, y - TRI[0])
        if l1 >= 0 and l2 >= 0 and l1 + l2 <= 1:
            continue
        cands = [_seg(x, TRI[0], TRI[1]), _seg(x, TRI[1], TRI[2]), _seg(x, TRI[0], TRI[2])]
        ref = min(cands, key=lambda q: np.linalg.norm(x - q))
        assert np.allclose(_cp(x)[0], ref, atol=1e-12)
        checked += 1
    assert checked > 500


def test_closest_point_beats_dense_sampling():
    rng = np.random.default_rng(4)
    u, v = np.meshgrid(np.linspace(0, 1, 121), np.linspace(0, 1, 121))
    keep = (u + v) <= 1
    S = (1 - u[keep] - v[keep])[:, None] * TRI[0] + u[keep][:, None] * TRI[1] + v[keep][:, None] * TRI[2]
    for _ in range(100):
        x = TRI.mean(0) + rng.normal(size=3)
        y = _cp(x)[0]
        d = np.linalg.norm(x - y)
        assert d <= np.linalg.norm(S - x, axis=1).min() + 1e-12
        # y lies in the triangle: non-negative barycentric coordinates
        M = np.column_stack([TRI[1] - TRI[0], TRI[2] - TRI[0], _normal()])
        l1, l2, off = np.linalg.solve(M, y - TRI[0])
        assert l1 >= -1e-12 and l2 >= -1e-12 and l1 + l2 <= 1 + 1e-12 and abs(off) < 1e-12


@pytest.fixture(scope="module")
def small_mesh():
    V, T = perturbed_icosphere(3, 0.15, 4)
    return V, T, geometry.TriMesh(V, T)


def test_trimesh_cp_matches_brute_force(small_mesh):
    V, T, S = small_mesh
    rng = np.random.default_rng(5)
    X = rng.normal(size=(400, 3))
    X = X / np.linalg.norm(X, axis=1)[:, None] * rng.uniform(0.6, 1.4, size=(400, 1))
    Y, tri = S.cp_tri(X)
    for q in range(len(X)):
        P = np.repeat(X[q][None], len(T), 0)
        Yb = closest_point_on_triangles(P, V[T[:, 0]], V[T[:, 1]], V[T[:, 2]])
        D = P - Yb
        d2 = (D[:, 0] * D[:, 0] + D[:, 1] * D[:, 1]) + D[:, 2] * D[:, 2]
        t = int(np.argmin(d2))            # first minimum = lowest triangle index
        assert tri[q] == t
        assert np.array_equal(Y[q], Yb[t])


def test_trimesh_dmax_only_drops_far_points(small_mesh):
    V, T, S = small_mesh
    rng = np.random.default_rng(6)
    X = rng.uniform(-1.3, 1.3, size=(3000, 3))
    Y, tri = S.cp_tri(X)
    Yd, trid = S.cp_tri(X, dmax=0.1)
    d = np.linalg.norm(X - Y, axis=1)
    near = d <= 0.1
    assert np.array_equal(trid[near], tri[near]) and np.array_equal(Yd[near], Y[near])
    assert np.all(trid[d > 0.1 * (1 + 1e-6)] == -1)


def test_face_normals_are_unit_and_outward(small_mesh):
    V, T, S = small_mesh
    assert np.allclose(np.linalg.norm(S.face_normal, axis=1), 1.0)
    ctr = (V[T[:, 0]] + V[T[:, 1]] + V[T[:, 2]]) / 3
    assert np.all(np.einsum("ij,ij->i", S.face_normal, ctr) > 0)


def test_icosphere_topology_and_sphere_approximation():
    for level in range(4):
        V, T = icosphere(level)
        assert len(T) == 20 * 4 ** level and len(V) == 10 * 4 ** level + 2
        assert np.allclose(np.linalg.norm(V, axis=1), 1.0)
    V, T = icosphere(4)
    S = geometry.TriMesh(V, T)
    rng = np.random.default_rng(7)
    X = rng.normal(size=(500, 3))
    X = X / np.linalg.norm(X, axis=1)[:, None] * rng.uniform(0.8, 1.2, size=(500, 1))
    Ymesh = S.cp(X)
    Ysph = geometry.Sphere(1.0).cp(X)
    # chordal error of a level-4 icosphere (edge ~0.077): sagitta e^2/8 plus in-plane shift
    assert np.abs(Ymesh - Ysph).max() < 0.01


def test_fine_icosphere_band_approaches_sphere_band():
    V, T = icosphere(5)
    h = 0.1
    n_mesh = band.count_active(geometry.TriMesh(V, T), h, 3)
    n_sph = band.count_active(geometry.Sphere(1.0), h, 3)
    assert abs(n_mesh - n_sph) / n_sph < 0.01


def _max_dihedral_curvature(V, T):
    """Discrete curvature estimate: angle between the normals of two faces sharing an edge
    divided by the distance of their centroids (maximum over edges)."""
    A, B, C = V[T[:, 0]], V[T[:, 1]], V[T[:, 2]]
    N = np.cross(B - A, C - A)
    N /= np.linalg.norm(N, axis=1)[:, None]
    ctr = (A + B + C) / 3
    owner = {}
    kmax = 0.0
    for f, (a, b, c) in enumerate(T):
        for e in ((a, b), (b, c), (c, a)):
            key = (min(e), max(e))
            if key in owner:
                g = owner[key]
                ang = math.acos(min(1.0, max(-1.0, float(N[f] @ N[g]))))
                kmax = max(kmax, ang / float(np.linalg.norm(ctr[f] - ctr[g])))
            else:
                owner[key] = f
    return kmax


def test_workload_mesh_band_width_condition():
    """The tube radius must stay below the reach 1/kappa_max of the surface (Sec. 2.1)."""
    wl = WORKLOADS["mesh_h001"]
    V, T = surface_mesh(wl)
    lam = band.default_lam_over_h(wl.p) * wl.h
    kmax = _max_dihedral_curvature(V, T)
    assert lam < 1.0 / kmax, (lam, kmax)


def test_mesh_small_ras_solve_matches_direct_solve():
    """One subdomain: RAS is the exact inverse, so one FGMRES step solves A u = f."""
    V, T = perturbed_icosphere(3, 0.15, 4)
    prob = problems.setup("trimesh", 0.0, 0.0, 0.1, 3, 1.0, 1, 1, "ras", verts=V, tris=T)
    f = np.random.default_rng(8).normal(size=prob.band.n_active)
    res = problems.solve(prob, f, 1e-12)
    import scipy.sparse.linalg as spla
    ref = spla.spsolve(prob.A.tocsc(), f)
    assert res.iterations == 1
    assert np.linalg.norm(res.x - ref) <= 1e-10 * np.linalg.norm(ref)


def test_mesh_oras_stationary_converges():
    V, T = perturbed_icosphere(3, 0.15, 4)
    prob = problems.setup("trimesh", 0.0, 0.0, 0.1, 3, 1.0, 4, 2, "oras", 4.0, 40.0,
                          verts=V, tris=T)
    f = np.random.default_rng(9).normal(size=prob.band.n_active)
    u, it, ok = schwarz.stationary_solve(prob.A, prob.M, f, 1e-8, 500)
    assert ok
    assert np.linalg.norm(f - prob.A @ u) <= 1e-8 * np.linalg.norm(f)
