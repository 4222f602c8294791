"""Triangulated surfaces through the C ABI against the oracle (needs a GB300).

Small case (perturbed icosphere, 1,280 triangles, h = 0.05, 8 subdomains, ORAS): every
entry of A x and M^{-1} r against the oracle, and the FGMRES solution.  Tolerances as in
test_gpu_parity.

Full size (81,920 triangles, h = 0.01, N_A ~ 9.4e5, 256 subdomains, FP32 factors, autotuned
solve as benchmarked): the whole oracle band takes minutes, so the oracle checks sampled
outputs one by one --
  * closest points and triangles of sampled nodes by a brute-force scan of every triangle
    (bit-exact) and their tube-test side (actives within lambda, ghosts beyond);
  * sampled rows of A x from the oracle's own closest points and barycentric weights;
  * the solve reaches the tolerance, and sampled entries of its residual f - A u agree
    with the oracle's row formula.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
import paper_1909_08734_gb300 as G  # noqa: E402
from oracle import interp, problems  # noqa: E402
from oracle.geometry import closest_point_on_triangles  # noqa: E402
from workloads import WORKLOADS, random_vector, rhs, surface_mesh  # noqa: E402

pytestmark = pytest.mark.gpu
EPS = np.finfo(float).eps


def _dev(x):
    return torch.tensor(np.ascontiguousarray(x), dtype=torch.float64, device="cuda")


@pytest.fixture(scope="module")
def small():
    wl = WORKLOADS["mesh_small"]
    V, T = surface_mesh(wl)
    band = G.cpm_build_band("trimesh", 0.0, 0.0, wl.h, wl.p, verts=V, tris=T)
    part = G.cpm_partition(band, wl.n_sub, None, wl.n_overlap)
    prob = problems.setup_workload(wl)
    return wl, band, part, prob


def test_mesh_apply_parity(small):
    wl, band, part, prob = small
    pc = G.oras_setup(band, part, wl.c, "ras", 0, 0, "fp64")
    x = random_vector(pc.n_active, 21)
    y = torch.empty(pc.n_active, dtype=torch.float64, device="cuda")
    G.cpm_op_apply(pc, _dev(x), y)
    ref = prob.A @ x
    assert np.all(np.abs(y.cpu().numpy() - ref) <= 64 * EPS * (abs(prob.A) @ np.abs(x)))


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-10), ("fp32", 1e-3)])
def test_mesh_preconditioner_parity(small, prec, tol):
    wl, band, part, prob = small
    pc = G.oras_setup(band, part, wl.c, "oras", wl.alpha, wl.alpha_x, prec)
    assert list(pc.local_sizes()) == [lp.n for lp in prob.lps]
    r = random_vector(pc.n_active, 22)
    z = torch.empty(pc.n_active, dtype=torch.float64, device="cuda")
    G.oras_apply(pc, _dev(r), z)
    G.oras_check_status(pc)
    ref = prob.M.apply(r)
    assert np.linalg.norm(z.cpu().numpy() - ref) / np.linalg.norm(ref) <= tol


def test_mesh_gmres_matches_oracle(small):
    wl, band, part, prob = small
    pc = G.oras_setup(band, part, wl.c, "oras", wl.alpha, wl.alpha_x, "fp64")
    u = torch.zeros(pc.n_active, dtype=torch.float64, device="cuda")
    res = G.cpm_gmres_solve(pc, _dev(prob.f), u, tol=1e-12)[0]
    ref = problems.solve(prob, prob.f, 1e-12)
    assert res["status"] == 0 and abs(res["iterations"] - ref.iterations) <= 1
    assert np.linalg.norm(u.cpu().numpy() - ref.x) / np.linalg.norm(ref.x) <= 1e-10


# ---------------------------------------------------------------- full size, sampled
class FullMesh:
    def __init__(self):
        wl = WORKLOADS["mesh_h001"]
        self.wl = wl
        self.V, self.T = surface_mesh(wl)
        self.band = G.cpm_build_band("trimesh", 0.0, 0.0, wl.h, wl.p, verts=self.V, tris=self.T)
        self.info = self.band.info()
        self.part = G.cpm_partition(self.band, wl.n_sub, None, wl.n_overlap)
        self.A = self.V[self.T[:, 0]]
        self.B = self.V[self.T[:, 1]]
        self.C = self.V[self.T[:, 2]]
        ijk = self.info["ijk"]
        self.index = {tuple(q): g for g, q in enumerate(map(tuple, ijk))}
        self.pc = None

    def brute_cp(self, x):
        """Oracle closest point over all triangles (ties: lowest index)."""
        P = np.repeat(np.asarray(x, dtype=np.float64)[None], len(self.T), 0)
        Y = closest_point_on_triangles(P, self.A, self.B, self.C)
        D = P - Y
        d2 = (D[:, 0] * D[:, 0] + D[:, 1] * D[:, 1]) + D[:, 2] * D[:, 2]
        t = int(np.argmin(d2))
        return Y[t], t

    def row(self, i, x):
        """(A x)_i and (|A| |x|)_i from the oracle's closest points and weights."""
        wl = self.wl
        h, p = wl.h, wl.p
        q = self.info["ijk"][i]
        diag = wl.c + 6.0 / (h * h)
        acc, mag = diag * x[i], abs(diag * x[i])
        off = interp.stencil_offsets(p)
        for d in ((-1, 0, 0), (1, 0, 0), (0, -1, 0), (0, 1, 0), (0, 0, -1), (0, 0, 1)):
            k = q + np.array(d)
            y, _ = self.brute_cp(k.astype(np.float64) * h)
            Bs, Wx, Wy, Wz = interp.point_weights(y[None], h, p)
            W = interp.tensor_weights(Wx, Wy, Wz)[0]
            cols = [self.index[tuple(Bs[0] + o)] for o in off]
            v = float(np.dot(W, x[cols]))
            acc -= v / (h * h)
            mag += float(np.dot(np.abs(W), np.abs(x[cols]))) / (h * h)
        return acc, mag

    def precond(self):
        if self.pc is None:
            wl = self.wl
            self.pc = G.oras_setup(self.band, self.part, wl.c, wl.method, wl.alpha, wl.alpha_x,
                                   wl.precision)
            G.oras_autotune(self.pc)
        return self.pc


@pytest.fixture(scope="module")
def full():
    F = FullMesh()
    yield F
    F.pc = None
    torch.cuda.empty_cache()


def test_full_mesh_band_sampled(full):
    inf = full.info
    na, ng = inf["n_active"], inf["n_ghost"]
    assert 9e5 < na < 1.1e6
    lam = inf["lambda"]
    rng = np.random.Generator(np.random.PCG64(31))
    sample = np.concatenate([rng.choice(na, 150, replace=False), na + rng.choice(ng, 50, replace=False)])
    for g in sample:
        x = inf["ijk"][g].astype(np.float64) * inf["h"]
        y, t = full.brute_cp(x)
        assert np.array_equal(inf["cp"][g], y) and inf["tri"][g] == t
        d = x - y
        dist = np.sqrt((d[0] * d[0] + d[1] * d[1]) + d[2] * d[2])
        assert (dist <= lam) == (g < na)


def test_full_mesh_apply_sampled_rows(full):
    pc = full.precond()
    n = pc.n_active
    x = random_vector(n, 32)
    y = torch.empty(n, dtype=torch.float64, device="cuda")
    G.cpm_op_apply(pc, _dev(x), y)
    Y = y.cpu().numpy()
    rng = np.random.Generator(np.random.PCG64(33))
    for i in rng.choice(n, 60, replace=False):
        ref, mag = full.row(i, x)
        assert abs(Y[i] - ref) <= 64 * EPS * mag, i


def test_full_mesh_solve(full):
    wl = full.wl
    pc = full.precond()
    n = pc.n_active
    f = rhs(wl, full.info["cp"][:n])
    u = torch.zeros(n, dtype=torch.float64, device="cuda")
    res = G.cpm_gmres_solve(pc, _dev(f), u, tol=wl.tol, restart=wl.restart, max_it=wl.max_it)[0]
    assert res["status"] == 0 and res["relres"] <= wl.tol
    U = u.cpu().numpy()
    au = torch.empty_like(u)
    G.cpm_op_apply(pc, u, au)
    r = f - au.cpu().numpy()
    assert np.linalg.norm(r) <= wl.tol * np.linalg.norm(f) * (1 + 1e-6)
    rng = np.random.Generator(np.random.PCG64(34))
    for i in rng.choice(n, 30, replace=False):
        ref, mag = full.row(i, U)
        assert abs((f[i] - ref) - r[i]) <= 64 * EPS * (mag + abs(f[i])), i
