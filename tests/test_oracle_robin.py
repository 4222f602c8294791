"""Pins of the ORAS local operator (Robin transmission rows) against the mathematics.

The oracle's Robin rows follow Sec. 5.2: T-rows interpolate at CP_{S_j}(x_i) (Eq. locCP) and are
scaled by 1 / (1 + alpha d.q) (Eq. robfo), with d.q = |d - (d.n) n| (Eq. naConorm).  These tests
check them against facts that do not come from the oracle's own code:

* Exact Robin data.  Eq. discRob with a nonzero right-hand side g (the condition
  du/dq + alpha u = g) gives u(x_i) = [u(CP_{S_j}(x_i)) + g d.q] / (1 + alpha d.q).  On the unit
  sphere u = xyz solves (c - Lap_S) u = (c + 12) u; for a spherical-cap subdomain the local
  problem with f = (c + 12) xyz and g = grad u . q + alpha u evaluated independently (analytic
  normal n = y at y = CP_{S_j}(x)) must reproduce u at the surface with first-order error in h,
  the order Table 1 reports for this discretisation, under reading R1 and under R3.
* The normal sits at CP_{S_j}(x_i): the oracle's d.q equals the analytic-normal value exactly.
* alpha -> infinity: every T-row with d.q > 0 vanishes, so under R3 the local problem is the
  Dirichlet transmission of Sec. 5.1 written with T_j = [0 I] and zero boundary values; the
  solution on Sigma_j equals that operator's, built here from the global E and the neighbour
  table.  It is not R_j A R_j^T: that keeps the extension rows of the boundary neighbours.
* R1 and R3 give different local matrices (boundary rows only), so comparing them is not vacuous.
* A planted mistake (the Robin weight doubled in the oracle's T-rows) destroys convergence.
"""
import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from oracle import band as band_mod
from oracle import geometry, interp, local, operator, partition
from workloads import random_vector

C = 1.0
ALPHA = 4.0


def _xyz(Y):
    return Y[:, 0] * Y[:, 1] * Y[:, 2]


def cap_problem(h, reading, alpha=ALPHA, zcut=0.3, n_overlap=2):
    """Unit sphere, subdomain 0 = actives whose CP has z > zcut (a spherical cap), overlap 2."""
    B = band_mod.build_band(geometry.make_surface("sphere", 1.0, 0.0), h, 3)
    E = interp.extension_matrix(B)
    labels = (B.cp[: B.n_active, 2] <= zcut).astype(np.int64)
    sub = partition.build_subdomain(B, E, labels, 0, n_overlap, reading == "R1")
    marks = partition.CrossMarks(B, partition.cross_point_nodes(B, labels), n_overlap)
    lp = local.oras_local(B, sub, C, alpha, 10 * alpha, marks, reading)
    return B, E, sub, lp


def analytic_dq(B, lp):
    X = B.coords(lp.bc_nodes)
    y = lp.bc_cp
    d = X - y
    n = y / np.linalg.norm(y, axis=1)[:, None]
    dperp = d - np.sum(d * n, axis=1)[:, None] * n
    return y, dperp, np.linalg.norm(dperp, axis=1)


def exact_data_error(h, reading):
    """Max error at the surface of the local solution with exact Robin data."""
    B, E, sub, lp = cap_problem(h, reading)
    U, n, ns = lp.unknowns, lp.n, lp.n_sigma
    y, dperp, dq = analytic_dq(B, lp)
    grad = np.stack([y[:, 1] * y[:, 2], y[:, 0] * y[:, 2], y[:, 0] * y[:, 1]], axis=1)
    # affine part of the boundary extension: g d.q / (1 + alpha d.q), with g d.q = grad u . dperp
    # + alpha u d.q (the conormal q = dperp / d.q)
    t = (np.sum(grad * dperp, axis=1) + lp.bc_alpha * _xyz(y) * dq) / (1.0 + lp.bc_alpha * dq)
    tn = np.zeros(B.n_nodes)
    tn[lp.bc_nodes] = t
    bc = np.zeros(B.n_nodes, bool)
    bc[lp.bc_nodes] = True
    ih2 = 1.0 / (h * h)
    b = (C + 12.0) * _xyz(B.cp[U])
    n_pde = n if reading == "R1" else ns          # rows with the 7-point Laplacian
    nb = B.nbr[U[:n_pde]]
    b[:n_pde] += ih2 * np.sum(np.where(bc[nb], tn[nb], 0.0), axis=1)
    if reading == "R3":                           # rows (c + 6/h^2) w - (6/h^2) (T w + t)
        b[ns:] += 6.0 * ih2 * tn[U[ns:]]
    w = spla.spsolve(lp.A.tocsc(), b)
    loc = np.full(B.n_active, -1)
    loc[U] = np.arange(n)
    cols, wts = interp.interpolation_rows(B, B.cp[U[:ns]])
    v = np.sum(wts * w[loc[cols]], axis=1)        # surface values at CP(x), x in Sigma_j
    return np.max(np.abs(v - _xyz(B.cp[U[:ns]])))


@pytest.mark.parametrize("reading", ["R1", "R3"])
def test_exact_robin_data_converges_at_first_order(reading):
    e1, e2 = exact_data_error(0.1, reading), exact_data_error(0.05, reading)
    assert e2 < 1e-2, (e1, e2)
    assert e1 / e2 > 1.5, (e1, e2)


def test_normal_at_the_subdomain_closest_point():
    B, E, sub, lp = cap_problem(0.1, "R1")
    _, _, dq = analytic_dq(B, lp)
    assert len(dq) > 100
    assert np.max(np.abs(dq - lp.bc_dq)) <= 1e-15


def test_alpha_infinity_is_dirichlet_transmission():
    h = 0.1
    B, E, sub, lp = cap_problem(h, "R3", alpha=1e16)
    assert np.all(lp.bc_dq > 0)
    S = sub.sigma
    ns = len(S)
    extended = np.zeros(B.n_nodes, bool)          # nodes extended by E: Sigma_j and its ghosts
    extended[S] = True
    extended[sub.ghost] = True
    nb = B.nbr[S]
    N = sp.csr_matrix((np.where(extended[nb], 1.0, 0.0).ravel(), (np.repeat(np.arange(ns), 6), nb.ravel())),
                      shape=(ns, B.n_nodes))
    D = (C + 6.0 / h**2) * sp.eye(ns) - (N @ E.tocsr()[:, S]) / h**2
    r = random_vector(B.n_active, 5)
    z_dir = spla.spsolve(D.tocsc(), r[S])
    z_loc = spla.spsolve(lp.A.tocsc(), lp.rhs(r))[:ns]
    assert np.max(np.abs(z_loc - z_dir)) <= 1e-12 * np.max(np.abs(z_dir))
    A = operator.cpm_matrix(B, E, C).tocsr()
    z_ras = spla.spsolve(A[S][:, S].tocsc(), r[S])
    assert np.max(np.abs(z_ras - z_dir)) > 1e-3 * np.max(np.abs(z_dir))


def test_r1_and_r3_local_matrices_differ():
    _, _, _, l1 = cap_problem(0.1, "R1")
    _, _, _, l3 = cap_problem(0.1, "R3")
    assert np.array_equal(l1.unknowns, l3.unknowns) and l1.n_sigma == l3.n_sigma
    dA = abs(l1.A - l3.A).sum(axis=1).A1
    ns = l1.n_sigma
    assert np.all(dA[:ns] <= 1e-9 * abs(l1.A).sum(axis=1).A1[:ns])   # Sigma_j rows agree
    assert np.all(dA[ns:] > 0)                                        # every boundary row differs


def test_planted_robin_weight_mistake_is_caught(monkeypatch):
    orig = local.robin_rows

    def doubled(band, sub, nodes, near_cross, alpha, alpha_x):
        return orig(band, sub, nodes, near_cross, 2 * alpha, 2 * alpha_x)[:2] + \
            orig(band, sub, nodes, near_cross, alpha, alpha_x)[2:]

    monkeypatch.setattr(local, "robin_rows", doubled)
    e1, e2 = exact_data_error(0.1, "R1"), exact_data_error(0.05, "R1")
    assert not (e2 < 1e-2 and e1 / e2 > 1.5), (e1, e2)
