"""Full-size parity of the benchmarked workloads (needs a GB300).

The unit sphere at h = 0.025 (N_A ~ 1.4e5, 64 subdomains, ORAS) and the torus R = 1, r = 0.4
at h = 0.0125 (N_A ~ 7.0e5, 512 random-weight subdomains, ORAS, BF16 factors) are run in the
configuration the benchmark times: autotuned solve schedule, CUDA-graph iterations.

What the oracle checks at this size:
  * operator apply: every entry against the oracle's sparse A (Eqs. impLapBel, simpleRAS),
    bound 64 eps (|A| |x|)_i;
  * preconditioner: every subdomain j, entry by entry; the oracle assembles A_j from the
    paper's local-operator definition (Eq. localOP, Robin rows Eq. robfo) in worker processes,
    solves it with SuperLU and compares z on the disjoint set of j, which M^{-1} writes from
    that subdomain alone (Eq. restCons);
  * solve: the true relative residual ||f - A u|| / ||f|| recomputed with the oracle's A.
"""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

torch = pytest.importorskip("torch")
import paper_1909_08734_gb300 as G  # noqa: E402
from oracle import band as band_mod  # noqa: E402
from oracle import geometry, interp, local, operator, partition  # noqa: E402
from workloads import WORKLOADS, leaf_weights, random_vector, rhs  # noqa: E402

pytestmark = pytest.mark.gpu
EPS = np.finfo(float).eps
# relative tolerance of one subdomain's z_j by factor precision (see test_gpu_parity)
LOCAL_TOL = {"fp64": 1e-10, "fp32": 1e-3, "bf16": 5e-2}


class Full:
    def __init__(self, name):
        wl = WORKLOADS[name]
        self.wl = wl
        w = leaf_weights(wl.n_sub, wl.weight_seed)
        self.band = G.cpm_build_band(wl.surface, wl.R, wl.r, wl.h, wl.p)
        self.part = G.cpm_partition(self.band, wl.n_sub, w, wl.n_overlap)
        surf = geometry.make_surface(wl.surface, wl.R, wl.r)
        self.B = band_mod.build_band(surf, wl.h, wl.p)
        self.E = interp.extension_matrix(self.B)
        self.A = operator.cpm_matrix(self.B, self.E, wl.c)
        self.labels = partition.rcb(self.B.cp[: self.B.n_active], wl.n_sub, w)
        self.marks = partition.CrossMarks(self.B, partition.cross_point_nodes(self.B, self.labels),
                                          wl.n_overlap)
        self.f = rhs(wl, self.B.cp[: self.B.n_active])
        self._pcs = {}

    def pc(self, prec):
        if prec not in self._pcs:
            wl = self.wl
            p = G.oras_setup(self.band, self.part, wl.c, wl.method, wl.alpha, wl.alpha_x, prec)
            G.oras_autotune(p)
            self._pcs[prec] = p
        return self._pcs[prec]

    def local_problem(self, j):
        wl = self.wl
        sub = partition.build_subdomain(self.B, self.E, self.labels, j, wl.n_overlap,
                                        wl.method == "oras")
        if wl.method == "ras":
            return local.ras_local(self.A, sub)
        return local.oras_local(self.B, sub, wl.c, wl.alpha, wl.alpha_x, self.marks, "R1")


@pytest.fixture(scope="module", params=["sphere_h0025", "torus_h00125"])
def full(request):
    F = Full(request.param)
    yield F
    F._pcs.clear()
    torch.cuda.empty_cache()


def _dev(x):
    return torch.tensor(np.ascontiguousarray(x), dtype=torch.float64, device="cuda")


def test_full_band_matches_oracle(full):
    info = full.band.info()
    assert info["n_active"] == full.B.n_active
    assert info["n_ghost"] == full.B.n_ghost
    assert np.array_equal(info["ijk"], full.B.ijk)


def test_full_apply_parity(full):
    pc = full.pc(full.wl.precision)
    n = pc.n_active
    X = random_vector(n, 11)
    y = torch.empty(n, dtype=torch.float64, device="cuda")
    G.cpm_op_apply(pc, _dev(X), y)
    ref = full.A @ X
    bound = 64 * EPS * (abs(full.A) @ np.abs(X))
    assert np.all(np.abs(y.cpu().numpy() - ref) <= bound)


def test_full_preconditioner_every_subdomain(full):
    """M^{-1} r entry by entry on the disjoint set of every subdomain (Eq. restCons: each entry
    comes from one local solve) against SuperLU on the oracle's A_j, for the benchmarked factor
    precision and for FP64: |z - z_ref| <= tol max|z_ref| per subdomain."""
    import os
    import oracle_local_pool
    wl = full.wl
    r = random_vector(full.B.n_active, 12)
    z = {}
    for prec in sorted({wl.precision, "fp64"}):
        pc = full.pc(prec)
        zz = torch.empty(pc.n_active, dtype=torch.float64, device="cuda")
        G.oras_apply(pc, _dev(r), zz)
        G.oras_check_status(pc)
        z[prec] = zz.cpu().numpy()
    sizes = np.asarray(full.pc(wl.precision).local_sizes())
    workers = max(1, min(16, (os.cpu_count() or 2) - 1))
    ref = oracle_local_pool.all_local_solutions(wl.name, r, wl.n_sub, workers)
    assert [t[0] for t in ref] == list(range(wl.n_sub))
    covered = np.zeros(full.B.n_active, dtype=np.int64)
    for j, n_j, own, zr in ref:
        assert n_j == sizes[j], j
        covered[own] += 1
        scale = np.max(np.abs(zr))
        for prec, zz in z.items():
            err = np.max(np.abs(zz[own] - zr))
            assert err <= LOCAL_TOL[prec] * scale, (prec, j, err / scale)
    assert np.all(covered == 1)                   # the disjoint sets partition the actives


def test_full_solve_true_residual(full):
    """The benchmarked solve reaches the tolerance in the oracle's own residual."""
    wl = full.wl
    pc = full.pc(wl.precision)
    u = torch.zeros(pc.n_active, dtype=torch.float64, device="cuda")
    res = G.cpm_gmres_solve(pc, _dev(full.f), u, tol=wl.tol, restart=wl.restart,
                            max_it=wl.max_it)[0]
    assert res["status"] == 0
    U = u.cpu().numpy()
    true = np.linalg.norm(full.f - full.A @ U) / np.linalg.norm(full.f)
    assert true <= wl.tol * (1 + 1e-6), true
    # both residuals carry cancellation error ~eps (|A||u|)_i ~ 1e-12 ||f|| at these h
    assert abs(true - res["relres"]) <= 1e-3 * wl.tol
    # the FP64-factor solve reaches the same solution up to cond(A) * 2 tol, with cond(A)
    # bounded by (c + 12 / h^2) / c (largest / smallest eigenvalue scale of c - Lap_h)
    pc64 = full.pc("fp64")
    u64 = torch.zeros_like(u)
    r64 = G.cpm_gmres_solve(pc64, _dev(full.f), u64, tol=wl.tol, restart=wl.restart,
                            max_it=wl.max_it)[0]
    assert r64["status"] == 0
    assert abs(res["iterations"] - r64["iterations"]) <= 3
    diff = np.linalg.norm(U - u64.cpu().numpy()) / np.linalg.norm(U)
    assert diff <= 2 * wl.tol * (wl.c + 12 / wl.h ** 2) / wl.c, diff
