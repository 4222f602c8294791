"""Pins for the oracle's partition, overlap, node sets and local operators (CPU only)."""
import math

import networkx as nx
import numpy as np
import pytest
import scipy.sparse.linalg as spla

from oracle import band, geometry, interp, local, operator, partition, problems


@pytest.fixture(scope="module")
def small():
    B = band.build_band(geometry.Sphere(1.0), 0.1, 3)
    E = interp.extension_matrix(B)
    A = operator.cpm_matrix(B, E, 1.0)
    return B, E, A


def _rcb_reference(points, idx, l0, l1, w, out):
    """Plain recursive bisection with python sorting (independent restatement)."""
    if l1 - l0 == 1:
        for i in idx:
            out[i] = l0
        return
    ext = [max(points[i][a] for i in idx) - min(points[i][a] for i in idx) for a in range(3)]
    axis = ext.index(max(ext))
    srt = sorted(idx, key=lambda i: (points[i][axis], i))
    PL = (l1 - l0) // 2
    nL = len(idx) * sum(w[l0:l0 + PL]) // sum(w[l0:l1])
    _rcb_reference(points, srt[:nL], l0, l0 + PL, w, out)
    _rcb_reference(points, srt[nL:], l0 + PL, l1, w, out)


@pytest.mark.parametrize("n_sub,weights", [(8, None), (6, None), (8, [300, 1000, 256, 700, 512, 999, 260, 800])])
def test_rcb_matches_reference(n_sub, weights):
    rng = np.random.default_rng(n_sub)
    pts = rng.uniform(-1, 1, (500, 3))
    pts[:40, 0] = 0.25                           # ties on a coordinate
    lab = partition.rcb(pts, n_sub, weights)
    ref = [None] * len(pts)
    w = [1] * n_sub if weights is None else weights
    _rcb_reference(pts.tolist(), list(range(len(pts))), 0, n_sub, w, ref)
    assert lab.tolist() == ref


def test_overlap_matches_networkx_bfs(small):
    B, E, A = small
    lab = partition.rcb(B.cp[:B.n_active], 8)
    G = nx.Graph()
    G.add_nodes_from(range(B.n_active))
    for a in range(B.n_active):
        for g in B.nbr[a]:
            if g < B.n_active:
                G.add_edge(a, int(g))
    for j in (0, 5):
        src = np.flatnonzero(lab == j).tolist()
        d = nx.multi_source_dijkstra_path_length(G, src, cutoff=3)
        sub = partition.build_subdomain(B, E, lab, j, 3, robin=True)
        assert sorted(d) == sub.sigma.tolist()
        assert sorted(k for k, v in d.items() if v == 3) == sub.last.tolist()


def test_node_sets_brute_force(small):
    B, E, A = small
    lab = partition.rcb(B.cp[:B.n_active], 8)
    sub = partition.build_subdomain(B, E, lab, 2, 2, robin=True)
    sig = set(sub.sigma.tolist())
    n_a = B.n_active
    Ecsr = E.tocsr()
    ghosts, bca = set(), set()
    for a in sig:
        for g in B.nbr[a]:
            g = int(g)
            if g >= n_a:
                ghosts.add(g)
            elif g not in sig:
                bca.add(g)
    for row in list(sig) + list(ghosts):
        for col in Ecsr.indices[Ecsr.indptr[row]:Ecsr.indptr[row + 1]]:
            if int(col) not in sig:
                bca.add(int(col))
    bcg = set()
    for a in bca:
        for g in B.nbr[a]:
            g = int(g)
            if g not in sig and g not in ghosts and g not in bca:
                bcg.add(g)
    assert sub.ghost.tolist() == sorted(ghosts)
    assert sub.bc_a.tolist() == sorted(bca)
    assert sub.bc_g.tolist() == sorted(bcg)


def test_cross_points_and_marks_brute_force(small):
    B, E, A = small
    lab = partition.rcb(B.cp[:B.n_active], 8)
    cross = partition.cross_point_nodes(B, lab)
    ref = []
    for a in range(B.n_active):
        others = {int(lab[g]) for g in B.nbr[a] if g < B.n_active and lab[g] != lab[a]}
        if len(others) >= 2:
            ref.append(a)
    assert cross.tolist() == ref and len(ref) > 0
    n_o = 2
    marks = partition.CrossMarks(B, cross, n_o)
    nodes = np.arange(0, B.n_nodes, 7)
    got = marks(nodes)
    C = B.ijk[cross]
    for q, g in zip(nodes, got):
        d2 = ((C - B.ijk[q]) ** 2).sum(1).min()
        assert g == (d2 <= (2 * n_o) ** 2)


def test_effective_boundary_cp_brute_force(small):
    B, E, A = small
    lab = partition.rcb(B.cp[:B.n_active], 8)
    sub = partition.build_subdomain(B, E, lab, 1, 2, robin=True)
    nodes = np.concatenate([sub.bc_a, sub.bc_g])[::5]
    y, gen = partition.effective_boundary_cp(B, sub, nodes)
    for q, yy, gg in zip(nodes, y, gen):
        x = B.ijk[q] * B.h
        best, bi = None, None
        for t in sub.last:                      # ascending tags: first minimum wins
            d = x - B.cp[t]
            d2 = (d[0] * d[0] + d[1] * d[1]) + d[2] * d[2]
            if best is None or d2 < best:
                best, bi = d2, t
        assert gg == bi and np.array_equal(yy, B.cp[bi])


def test_conormal_dot_product_identity():
    # Eq. naConorm: q = d_perp / |d_perp|, so d . q = |d_perp|; d parallel to n gives 0
    rng = np.random.default_rng(3)
    for _ in range(100):
        d = rng.standard_normal(3)
        n = rng.standard_normal(3)
        n /= np.linalg.norm(n)
        dp = d - (d @ n) * n
        q = dp / np.linalg.norm(dp)
        assert abs(d @ q - np.linalg.norm(dp)) < 1e-14 * (1 + np.linalg.norm(d))
        assert abs(q @ n) < 1e-14
    n = np.array([0.0, 0.6, 0.8])
    d = 0.3 * n
    assert np.linalg.norm(d - (d @ n) * n) < 1e-16


def test_ras_local_is_restriction(small):
    B, E, A = small
    lab = partition.rcb(B.cp[:B.n_active], 8)
    sub = partition.build_subdomain(B, E, lab, 3, 2, robin=False)
    lp = local.ras_local(A, sub)
    Ad = A.toarray()
    assert np.array_equal(lp.A.toarray(), Ad[np.ix_(sub.sigma, sub.sigma)])


@pytest.mark.parametrize("method", ["ras", "oras"])
def test_one_subdomain_is_direct_solve(method):
    P = problems.setup("sphere", 1.0, 0.0, 0.1, 3, 1.0, 1, 2, method)
    assert P.lps[0].n == P.band.n_active
    f = np.random.default_rng(0).standard_normal(P.band.n_active)
    ud = spla.spsolve(P.A.tocsc(), f)
    res = problems.solve(P, f, 1e-12)
    assert res.iterations == 1
    assert np.linalg.norm(res.x - ud) <= 1e-10 * np.linalg.norm(ud)


def test_ras_full_overlap_is_exact_inverse():
    # overlap wider than the band: every Sigma_j = Sigma_A, so M^{-1} = A^{-1}
    P = problems.setup("sphere", 1.0, 0.0, 0.2, 3, 1.0, 4, 40, "ras")
    assert all(lp.n == P.band.n_active for lp in P.lps)
    r = np.random.default_rng(2).standard_normal(P.band.n_active)
    assert np.allclose(P.M.apply(r), spla.spsolve(P.A.tocsc(), r), rtol=0, atol=1e-10)


@pytest.mark.parametrize("reading", ["R1", "R3"])
def test_oras_converges_to_direct_solution(reading):
    P = problems.setup("sphere", 1.0, 0.0, 0.1, 3, 1.0, 8, 2, "oras", 4.0, 40.0, reading=reading)
    Y = P.band.cp[:P.band.n_active]
    f = 13.0 * Y[:, 0] * Y[:, 1] * Y[:, 2]
    res = problems.solve(P, f, 1e-11)
    ud = spla.spsolve(P.A.tocsc(), f)
    assert res.converged
    assert np.linalg.norm(res.x - ud) <= 1e-8 * np.linalg.norm(ud)


def test_robin_rows_scaling_limits(small):
    B, E, A = small
    lab = partition.rcb(B.cp[:B.n_active], 8)
    sub = partition.build_subdomain(B, E, lab, 4, 2, robin=True)
    cross = partition.cross_point_nodes(B, lab)
    marks = partition.CrossMarks(B, cross, 2)
    nodes = np.concatenate([sub.bc_a, sub.bc_g])
    c0, w0, y, gen, dq, a0 = local.robin_rows(B, sub, nodes, marks, 0.0, 0.0)
    # alpha = 0: the T-row is plain interpolation at CP_{S_j} (sums to one)
    assert np.abs(w0.sum(1) - 1.0).max() < 1e-14
    c1, w1, _, _, dq1, a1 = local.robin_rows(B, sub, nodes, marks, 4.0, 40.0)
    # Eq. robfo: scale 1 / (1 + alpha d.q), alpha_x exactly where the cross marks say
    assert np.allclose(w1.sum(1), 1.0 / (1.0 + a1 * dq1), rtol=1e-14)
    assert np.array_equal(a1 == 40.0, marks(nodes))
    assert np.all(dq1 >= 0) and np.all(dq1 <= np.linalg.norm(B.coords(nodes) - y, axis=1) + 1e-15)


def test_dense_and_sparse_local_lu_agree(small):
    P = problems.setup("sphere", 1.0, 0.0, 0.1, 3, 1.0, 8, 2, "oras", 4.0, 40.0)
    from oracle import schwarz
    Md = schwarz.Schwarz(P.lps, P.band.n_active, dense=True)
    r = np.random.default_rng(5).standard_normal(P.band.n_active)
    z1, z2 = P.M.apply(r), Md.apply(r)
    assert np.linalg.norm(z1 - z2) <= 1e-11 * np.linalg.norm(z1)


# ---------------------------------------------------------------- interface alignment
def _align_brute(band, labels, passes):
    """Sec. 3.2 restated with python loops and a dictionary of grid points."""
    lab = [int(x) for x in labels]
    n_a, h = band.n_active, band.h
    where = {tuple(int(v) for v in band.ijk[g]): g for g in range(n_a)}
    offs = [(-1, 0, 0), (1, 0, 0), (0, -1, 0), (0, 1, 0), (0, 0, -1), (0, 0, 1)]
    for _ in range(passes):
        new = list(lab)
        for g in range(n_a):
            i, j, k = (int(v) for v in band.ijk[g])
            nbl = [lab[where[(i + a, j + b, k + c)]] for a, b, c in offs if (i + a, j + b, k + c) in where]
            if all(l == lab[g] for l in nbl):
                continue
            near = tuple(int(math.floor(float(band.cp[g][a]) / h + 0.5)) for a in range(3))
            if near in where:
                new[g] = lab[where[near]]
        lab = new
    return np.array(lab)


def test_alignment_matches_brute_force_and_keeps_invariants():
    B = band.build_band(geometry.Sphere(1.0), 0.2, 2)
    lab0 = partition.rcb(B.cp[:B.n_active], 5)
    for passes in (1, 3):
        lab = partition.align_interfaces(B, lab0, passes)
        assert np.array_equal(lab, _align_brute(B, lab0, passes))
        assert set(np.unique(lab)) == set(range(5))
    # one pass changes only nodes that were interface nodes before it
    lab1 = partition.align_interfaces(B, lab0, 1)
    nb = B.nbr
    act = nb < B.n_active
    iface = np.any(act & (np.where(act, lab0[np.minimum(nb, B.n_active - 1)], -1) != lab0[:, None]), axis=1)
    assert np.all(iface[lab1 != lab0])


def test_alignment_reduces_misaligned_interface_nodes():
    """After p + 1 passes fewer interface nodes disagree with the label of the grid node
    nearest to their closest point (the quantity the passes drive down)."""
    B = band.build_band(geometry.Torus(1.0, 0.4), 0.05, 2)
    n_a = B.n_active
    near = B.lookup(np.floor(B.cp[:n_a] / B.h + 0.5).astype(np.int64))

    def misaligned(lab):
        act = B.nbr < n_a
        nl = np.where(act, lab[np.minimum(B.nbr, n_a - 1)], -1)
        iface = np.any(act & (nl != lab[:, None]), axis=1)
        return int(np.sum(iface & (lab[near] != lab)))

    lab0 = partition.rcb(B.cp[:n_a], 8)
    lab3 = partition.align_interfaces(B, lab0, 3)
    assert misaligned(lab3) < misaligned(lab0)

