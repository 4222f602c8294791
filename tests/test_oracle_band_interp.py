"""Pins for the oracle's band, extension matrix E and operator A (CPU only).

Each check compares the oracle with something other than itself: the paper's printed
active counts, a Vandermonde solve, monomials, a brute-force neighbour scan, spherical
harmonics and second-order convergence.
"""
import math
import os

import numpy as np
import pytest
import scipy.sparse.linalg as spla

from oracle import band, geometry, interp, operator

GOLD = os.path.join(os.path.dirname(__file__), "golden", "paper_band_counts.txt")


def _printed_counts():
    rows = []
    for line in open(GOLD):
        if line.strip() and not line.startswith("#"):
            inv, n = line.split()
            rows.append((int(inv), int(n)))
    return rows


@pytest.mark.parametrize("inv_h,n_a", _printed_counts())
def test_band_reproduces_printed_sphere_counts(inv_h, n_a):
    # Secs. 6.2 and 6.6: unit sphere, p = 2 (tri-quadratic)
    assert band.count_active(geometry.Sphere(1.0), 1.0 / inv_h, 2) == n_a


def test_band_radius_reading_interval():
    # the default radius lies in the interval that reproduces every printed count
    assert 2.60641 < band.default_lam_over_h(2) < 2.60699


def test_band_brute_force_small():
    s = geometry.Sphere(1.0)
    h, p = 0.25, 3
    B = band.build_band(s, h, p)
    lam = band.default_lam_over_h(p) * h
    # brute force over a big box with python loops
    act = []
    for i in range(-10, 11):
        for j in range(-10, 11):
            for k in range(-10, 11):
                x = np.array([i * h, j * h, k * h])
                r = math.sqrt((x[0] * x[0] + x[1] * x[1]) + x[2] * x[2])
                if r == 0:
                    continue
                y = x / r
                d = x - y
                if math.sqrt((d[0] * d[0] + d[1] * d[1]) + d[2] * d[2]) <= lam:
                    act.append((i, j, k))
    assert [tuple(v) for v in B.ijk[:B.n_active]] == sorted(act)
    aset = set(act)
    ghosts = set()
    for (i, j, k) in act:
        for d in [(-1, 0, 0), (1, 0, 0), (0, -1, 0), (0, 1, 0), (0, 0, -1), (0, 0, 1)]:
            q = (i + d[0], j + d[1], k + d[2])
            if q not in aset:
                ghosts.add(q)
    assert [tuple(v) for v in B.ijk[B.n_active:]] == sorted(ghosts)
    # neighbour table
    for a in range(B.n_active):
        for m, off in enumerate(band.NBR_OFFSETS):
            assert tuple(B.ijk[B.nbr[a, m]]) == tuple(B.ijk[a] + off)


def test_torus_cp_is_on_surface_and_nearest():
    t = geometry.Torus(1.0, 0.4)
    rng = np.random.default_rng(0)
    X = rng.uniform(-1.5, 1.5, size=(200, 3))
    X[:, 2] *= 0.4
    Y = t.cp(X)
    rho = np.sqrt(Y[:, 0] ** 2 + Y[:, 1] ** 2)
    assert np.allclose((rho - 1.0) ** 2 + Y[:, 2] ** 2, 0.16, atol=1e-12)
    # nearest: compare with a dense parametric sampling of the torus
    th, ph = np.meshgrid(np.linspace(0, 2 * np.pi, 721), np.linspace(0, 2 * np.pi, 721))
    S = np.stack([(1 + 0.4 * np.cos(ph)) * np.cos(th), (1 + 0.4 * np.cos(ph)) * np.sin(th),
                  0.4 * np.sin(ph)], -1).reshape(-1, 3)
    for x, y in zip(X[:20], Y[:20]):
        dmin = np.sqrt(((S - x) ** 2).sum(1)).min()
        assert np.linalg.norm(x - y) <= dmin + 1e-9


@pytest.mark.parametrize("p", [2, 3])
def test_barycentric_weights_match_vandermonde(p):
    rng = np.random.default_rng(p)
    t = rng.uniform(0.0, p, 50)
    W = interp.bary_weights_1d(t, p)
    nodes = np.arange(p + 1, dtype=float)
    V = np.vander(nodes, p + 1, increasing=True)          # V[m, e] = m^e
    for ti, wi in zip(t, W):
        # weights l with sum_m l_m m^e = t^e  <=>  V^T l = (t^e)
        ref = np.linalg.solve(V.T, ti ** np.arange(p + 1))
        assert np.allclose(wi, ref, atol=1e-13)


def test_barycentric_exact_node_is_delta():
    W = interp.bary_weights_1d(np.array([0.0, 1.0, 2.0, 3.0]), 3)
    assert np.array_equal(W, np.eye(4))
    # a closest point exactly on a grid node (binary-exact h) gives a unit-weight row
    B, Wx, Wy, Wz = interp.point_weights(np.array([[0.25, 0.5, 0.375]]), 0.125, 3)
    w = interp.tensor_weights(Wx, Wy, Wz)[0]
    assert np.count_nonzero(w) == 1 and w.max() == 1.0
    assert np.array_equal(B[0] + np.array([1, 1, 1]), [2, 4, 3])


@pytest.fixture(scope="module")
def small_sphere():
    B = band.build_band(geometry.Sphere(1.0), 0.1, 3)
    E = interp.extension_matrix(B)
    return B, E


def test_extension_rows_sum_to_one(small_sphere):
    B, E = small_sphere
    assert np.abs(np.asarray(E.sum(axis=1)).ravel() - 1.0).max() < 1e-14


@pytest.mark.parametrize("p", [2, 3])
def test_extension_reproduces_tensor_polynomials(p):
    B = band.build_band(geometry.Sphere(1.0), 0.1, p)
    E = interp.extension_matrix(B)
    X = B.coords()[:B.n_active]
    Y = B.cp
    for a in range(p + 1):
        for b in range(p + 1):
            for c in range(p + 1):
                u = X[:, 0] ** a * X[:, 1] ** b * X[:, 2] ** c
                ref = Y[:, 0] ** a * Y[:, 1] ** b * Y[:, 2] ** c
                assert np.abs(E @ u - ref).max() < 1e-12, (a, b, c)


def test_extension_stencil_error_when_band_too_thin():
    s = geometry.Sphere(1.0)
    B = band.build_band(s, 0.1, 3, lam_over_h=1.0)
    with pytest.raises(interp.StencilError):
        interp.extension_matrix(B)


def test_operator_maps_constants_to_c(small_sphere):
    B, E = small_sphere
    for c in (1.0, 10.0):
        A = operator.cpm_matrix(B, E, c)
        y = A @ np.ones(B.n_active)
        assert np.abs(y - c).max() < 1e-12 * (6.0 / B.h ** 2)


def test_operator_matrix_free_equals_assembled(small_sphere):
    B, E = small_sphere
    A = operator.cpm_matrix(B, E, 1.0)
    x = np.random.default_rng(1).standard_normal(B.n_active)
    assert np.allclose(operator.apply(B, E, 1.0, x), A @ x, rtol=0, atol=1e-9)


def _xyz_errors(h, construction="tube"):
    B = (band.build_band(geometry.Sphere(1.0), h, 3) if construction == "tube"
         else band.build_band_algorithmic(geometry.Sphere(1.0), h, 3))
    E = interp.extension_matrix(B)
    c = 1.0
    A = operator.cpm_matrix(B, E, c)
    Y = B.cp[:B.n_active]
    u = Y[:, 0] * Y[:, 1] * Y[:, 2]
    ud = spla.spsolve(A.tocsc(), (c + 12.0) * u)
    at_cp = E[:B.n_active] @ ud                  # discrete solution carried to the surface
    return np.abs(at_cp - u).max(), np.abs(ud - u).max()


def test_xyz_eigenfunction_second_order():
    # u = xyz is an l = 3 spherical harmonic: (c - Lap_S) u = (c + 12) u, so the discrete
    # solution of A u_h = (c + 12) xyz(CP) must approach xyz(CP) at second order in h.
    # (The residual A u - (c+12) u itself is only O(h) at band nodes off the surface, where
    # Lap(u o CP) = Lap_S u / rho^2 on a sphere of radius rho.)
    s1, e1 = _xyz_errors(0.2)
    s2, e2 = _xyz_errors(0.1)
    s3, e3 = _xyz_errors(0.05)
    assert s1 / s2 > 2.7 and s2 / s3 > 3.3
    assert e1 / e2 > 4.0 and e2 / e3 > 4.0
    assert s3 < 1e-4


# ---------------------------------------------------------------- algorithmic band
@pytest.mark.parametrize("surf,h,p", [(geometry.Sphere(1.0), 0.1, 3), (geometry.Torus(1.0, 0.4), 0.1, 2)])
def test_algorithmic_band_is_the_minimal_interpolation_closure(surf, h, p):
    A = band.build_band_algorithmic(surf, h, p)
    actives = set(map(tuple, A.ijk[:A.n_active].tolist()))
    # closed: every stencil of CP(x), x active or ghost, is active
    cols, _ = interp.interpolation_rows(A, A.cp)
    assert cols.min() >= 0 and cols.max() < A.n_active
    # minimal: every active node is a seed node (within h of the surface) or used by a stencil
    seed = set(map(tuple, band.active_nodes(surf, h, p, 1.0)[0].tolist()))
    used = set(map(tuple, A.ijk[np.unique(cols)].tolist()))
    assert actives == seed | used
    # and it sits inside the default tube band
    T = band.build_band(surf, h, p)
    assert actives <= set(map(tuple, T.ijk[:T.n_active].tolist()))
    assert A.n_active < T.n_active


def test_algorithmic_band_keeps_second_order():
    # same surface error as the tube band's at h = 0.2, 0.1 (ratio > 2.7, i.e. order > 1.4
    # in the pre-asymptotic range where the tube band shows the same ratio)
    s1, _ = _xyz_errors(0.2, "algorithmic")
    s2, _ = _xyz_errors(0.1, "algorithmic")
    t2, _ = _xyz_errors(0.1)
    assert s1 / s2 > 2.7 and s2 < 2.0 * t2
