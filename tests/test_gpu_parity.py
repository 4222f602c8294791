"""GPU parity through the C ABI against the CPU FP64 oracle (needs a GB300).

Tolerances follow from the arithmetic:
  operator apply  : each y_i is a sum of ~400 FP64 products, so
                    |y_gpu - y_ref| <= 64 eps (|A| |x|)_i.
  M^{-1} r, FP64  : both sides solve every A_j with a backward-stable LU, so they agree to
                    ~cond(A_j) eps; cond(A_j) <= 1e5 here, bound 1e-10 relative.
  M^{-1} r, FP32  : factor and solve in FP32, ~cond(A_j) 2^-24 relative -> 1e-3.
  M^{-1} r, BF16  : factors stored in BF16 (8-bit mantissa) -> 5e-2.
  GMRES, FP64     : converged to 1e-12, solution within 1e-10 relative of the oracle's.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
import paper_1909_08734_gb300 as G  # noqa: E402
from oracle import krylov, problems  # noqa: E402
from workloads import random_vector  # noqa: E402

pytestmark = pytest.mark.gpu
EPS = np.finfo(float).eps


def _dev(x):
    return torch.tensor(np.ascontiguousarray(x), dtype=torch.float64, device="cuda")


@pytest.fixture(scope="module")
def sphere_small():
    h, c = 0.1, 1.0
    band = G.cpm_build_band("sphere", 1.0, 0.0, h, 3)
    part = G.cpm_partition(band, 8, None, 2)
    oras = problems.setup("sphere", 1.0, 0.0, h, 3, c, 8, 2, "oras", 4.0, 40.0)
    ras = problems.setup("sphere", 1.0, 0.0, h, 3, c, 8, 2, "ras")
    return band, part, oras, ras, c


@pytest.fixture(scope="module")
def torus_uneven():
    h, c = 0.05, 10.0
    w = np.array([256, 1024, 300, 500, 999, 700, 260, 800, 400, 410, 420, 1000, 256, 257, 900, 333])
    band = G.cpm_build_band("torus", 1.0, 0.4, h, 3)
    part = G.cpm_partition(band, 16, w, 2)
    oras = problems.setup("torus", 1.0, 0.4, h, 3, c, 16, 2, "oras", 4.0, 40.0, leaf_weights=w)
    return band, part, oras, c


@pytest.fixture(scope="module")
def sphere_p2():
    # the paper's discretisation (Sec. 6): tri-quadratic interpolation, overlap 4,
    # alpha = 4 and alpha_x = 40 (Secs. 6.5, 6.6)
    h, c = 0.1, 1.0
    band = G.cpm_build_band("sphere", 1.0, 0.0, h, 2)
    part = G.cpm_partition(band, 8, None, 4)
    oras = problems.setup("sphere", 1.0, 0.0, h, 2, c, 8, 4, "oras", 4.0, 40.0)
    return band, part, oras, c


def test_p2_apply_preconditioner_and_solve(sphere_p2):
    band, part, oras, c = sphere_p2
    assert band.info()["n_active"] == oras.band.n_active
    pc = G.oras_setup(band, part, c, "oras", 4.0, 40.0, "fp64")
    n = pc.n_active
    x = random_vector(n, 31)
    y = torch.empty(n, dtype=torch.float64, device="cuda")
    G.cpm_op_apply(pc, _dev(x), y)
    bound = 64 * EPS * (abs(oras.A) @ np.abs(x))
    assert np.all(np.abs(y.cpu().numpy() - oras.A @ x) <= bound)
    r = random_vector(n, 32)
    z = torch.empty_like(y)
    G.oras_apply(pc, _dev(r), z)
    G.oras_check_status(pc)
    ref = oras.M.apply(r)
    assert np.linalg.norm(z.cpu().numpy() - ref) <= 1e-10 * np.linalg.norm(ref)
    cp = band.info()["cp"][:n]
    f = (c + 12.0) * cp[:, 0] * cp[:, 1] * cp[:, 2]
    u = torch.zeros(n, dtype=torch.float64, device="cuda")
    res = G.cpm_gmres_solve(pc, _dev(f), u, tol=1e-12)[0]
    sol = problems.solve(oras, f, 1e-12)
    assert res["status"] == 0 and abs(res["iterations"] - sol.iterations) <= 1
    assert np.linalg.norm(u.cpu().numpy() - sol.x) <= 1e-10 * np.linalg.norm(sol.x)


@pytest.mark.parametrize("prec,tol", [("fp32", 1e-3), ("bf16", 5e-2)])
def test_p2_low_precision_preconditioner(sphere_p2, prec, tol):
    band, part, oras, c = sphere_p2
    pc = G.oras_setup(band, part, c, "oras", 4.0, 40.0, prec)
    r = random_vector(pc.n_active, 33)
    z = torch.empty(pc.n_active, dtype=torch.float64, device="cuda")
    G.oras_apply(pc, _dev(r), z)
    G.oras_check_status(pc)
    ref = oras.M.apply(r)
    assert np.linalg.norm(z.cpu().numpy() - ref) <= tol * np.linalg.norm(ref)


def test_operator_apply_parity(sphere_small):
    band, part, oras, ras, c = sphere_small
    pc = G.oras_setup(band, part, c, "ras", 0, 0, "fp64")
    n = pc.n_active
    X = np.stack([random_vector(n, s) for s in (1, 2, 3)])
    x = _dev(X.ravel())
    y = torch.empty_like(x)
    G.cpm_op_apply(pc, x, y, nrhs=3)
    Y = y.cpu().numpy().reshape(3, n)
    absA = abs(oras.A)
    for r in range(3):
        ref = oras.A @ X[r]
        bound = 64 * EPS * (absA @ np.abs(X[r])) + 1e-300
        assert np.all(np.abs(Y[r] - ref) <= bound)


def test_operator_maps_constants_to_c(torus_uneven):
    band, part, oras, c = torus_uneven
    pc = G.oras_setup(band, part, c, "ras", 0, 0, "fp64")
    x = torch.ones(pc.n_active, dtype=torch.float64, device="cuda")
    y = torch.empty_like(x)
    G.cpm_op_apply(pc, x, y)
    h = band.info()["h"]
    assert torch.max(torch.abs(y - c)).item() <= 64 * EPS * (c + 12.0 / h ** 2)


@pytest.mark.parametrize("method", ["ras", "oras"])
def test_preconditioner_fp64_parity(sphere_small, method):
    band, part, oras, ras, c = sphere_small
    P = oras if method == "oras" else ras
    pc = G.oras_setup(band, part, c, method, 4.0, 40.0, "fp64")
    assert list(pc.local_sizes()) == [lp.n for lp in P.lps]
    r = random_vector(pc.n_active, 7)
    z = torch.empty(pc.n_active, dtype=torch.float64, device="cuda")
    G.oras_apply(pc, _dev(r), z)
    G.oras_check_status(pc)
    ref = P.M.apply(r)
    err = np.linalg.norm(z.cpu().numpy() - ref) / np.linalg.norm(ref)
    assert err <= 1e-10, err


def test_preconditioner_fp64_parity_uneven_torus(torus_uneven):
    band, part, oras, c = torus_uneven
    pc = G.oras_setup(band, part, c, "oras", 4.0, 40.0, "fp64")
    r = random_vector(pc.n_active, 8)
    z = torch.empty(pc.n_active, dtype=torch.float64, device="cuda")
    for _ in range(3):                       # repeated launches reuse the flags (epochs)
        G.oras_apply(pc, _dev(r), z)
    G.oras_check_status(pc)
    ref = oras.M.apply(r)
    err = np.linalg.norm(z.cpu().numpy() - ref) / np.linalg.norm(ref)
    assert err <= 1e-10, err


@pytest.mark.parametrize("prec,tol", [("fp32", 1e-3), ("bf16", 5e-2)])
def test_preconditioner_low_precision(sphere_small, prec, tol):
    band, part, oras, ras, c = sphere_small
    pc = G.oras_setup(band, part, c, "oras", 4.0, 40.0, prec)
    r = random_vector(pc.n_active, 9)
    z = torch.empty(pc.n_active, dtype=torch.float64, device="cuda")
    G.oras_apply(pc, _dev(r), z)
    G.oras_check_status(pc)
    ref = oras.M.apply(r)
    err = np.linalg.norm(z.cpu().numpy() - ref) / np.linalg.norm(ref)
    assert err <= tol, err


@pytest.mark.parametrize("use_graph", [True, False])
def test_gmres_fp64_matches_oracle(sphere_small, use_graph):
    band, part, oras, ras, c = sphere_small
    pc = G.oras_setup(band, part, c, "oras", 4.0, 40.0, "fp64")
    cp = band.info()["cp"][: pc.n_active]
    f = (c + 12.0) * cp[:, 0] * cp[:, 1] * cp[:, 2]
    u = torch.zeros(pc.n_active, dtype=torch.float64, device="cuda")
    res = G.cpm_gmres_solve(pc, _dev(f), u, tol=1e-12, use_graph=use_graph)[0]
    ref = problems.solve(oras, f, 1e-12)
    assert res["status"] == 0 and res["relres"] <= 1e-12
    assert abs(res["iterations"] - ref.iterations) <= 1
    err = np.linalg.norm(u.cpu().numpy() - ref.x) / np.linalg.norm(ref.x)
    assert err <= 1e-10, err


def test_gmres_kth_iterate_matches_oracle(sphere_small):
    band, part, oras, ras, c = sphere_small
    pc = G.oras_setup(band, part, c, "ras", 0, 0, "fp64")
    f = random_vector(pc.n_active, 11)
    for k in (1, 5, 12):
        u = torch.zeros(pc.n_active, dtype=torch.float64, device="cuda")
        res = G.cpm_gmres_solve(pc, _dev(f), u, tol=1e-30, max_it=k, raise_on_failure=False)[0]
        assert res["iterations"] == k and res["status"] == G._capi.CPM_ERR_NOT_CONVERGED
        ref = krylov.fgmres(lambda x: ras.A @ x, ras.M.apply, f, 1e-30, 50, 1000, stop_after=k)
        err = np.linalg.norm(u.cpu().numpy() - ref.x) / np.linalg.norm(ref.x)
        assert err <= 1e-11, (k, err)


def test_gmres_restarts(sphere_small):
    band, part, oras, ras, c = sphere_small
    pc = G.oras_setup(band, part, c, "ras", 0, 0, "fp64")
    f = random_vector(pc.n_active, 12)
    u = torch.zeros(pc.n_active, dtype=torch.float64, device="cuda")
    res = G.cpm_gmres_solve(pc, _dev(f), u, tol=1e-10, restart=5, max_it=500)[0]
    ref = krylov.fgmres(lambda x: ras.A @ x, ras.M.apply, f, 1e-10, 5, 500)
    assert res["status"] == 0 and abs(res["iterations"] - ref.iterations) <= 2
    err = np.linalg.norm(u.cpu().numpy() - ref.x) / np.linalg.norm(ref.x)
    assert err <= 1e-8, err


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_gmres_mixed_reaches_tolerance(torus_uneven, prec):
    band, part, oras, c = torus_uneven
    pc = G.oras_setup(band, part, c, "oras", 4.0, 40.0, prec)
    f = random_vector(pc.n_active, 13)
    u = torch.zeros(pc.n_active, dtype=torch.float64, device="cuda")
    res = G.cpm_gmres_solve(pc, _dev(f), u, tol=1e-8)[0]
    assert res["status"] == 0 and res["relres"] <= 1e-8
    ref = problems.solve(oras, f, 1e-12)
    err = np.linalg.norm(u.cpu().numpy() - ref.x) / np.linalg.norm(ref.x)
    assert err <= 1e-6, err


def test_zero_rhs_and_multi_rhs(sphere_small):
    band, part, oras, ras, c = sphere_small
    pc = G.oras_setup(band, part, c, "ras", 0, 0, "fp64")
    n = pc.n_active
    F = np.stack([np.zeros(n), random_vector(n, 14)])
    u = torch.zeros(2 * n, dtype=torch.float64, device="cuda")
    res = G.cpm_gmres_solve(pc, _dev(F.ravel()), u, nrhs=2, tol=1e-10)
    assert res[0]["status"] == 0 and res[0]["iterations"] == 0
    assert torch.count_nonzero(u[:n]).item() == 0
    assert res[1]["status"] == 0 and res[1]["relres"] <= 1e-10


def test_one_subdomain_is_direct_solve():
    band = G.cpm_build_band("sphere", 1.0, 0.0, 0.2, 3)
    part = G.cpm_partition(band, 1, None, 2)
    pc = G.oras_setup(band, part, 1.0, "oras", 4.0, 40.0, "fp64")
    P = problems.setup("sphere", 1.0, 0.0, 0.2, 3, 1.0, 1, 2, "oras")
    f = random_vector(pc.n_active, 15)
    u = torch.zeros(pc.n_active, dtype=torch.float64, device="cuda")
    res = G.cpm_gmres_solve(pc, _dev(f), u, tol=1e-12)[0]
    assert res["iterations"] == 1
    import scipy.sparse.linalg as spla
    ud = spla.spsolve(P.A.tocsc(), f)
    assert np.linalg.norm(u.cpu().numpy() - ud) <= 1e-10 * np.linalg.norm(ud)


def test_solve_schedules_agree(torus_uneven):
    # every schedule of the batched solve computes the same M^{-1} r up to rounding order
    band, part, oras, c = torus_uneven
    pc = G.oras_setup(band, part, c, "oras", 4.0, 40.0, "fp32")
    r = _dev(random_vector(pc.n_active, 16))
    z0 = torch.empty_like(r)
    G.oras_apply(pc, r, z0)
    for knobs in ({"kseg": 1}, {"kseg": 3, "prefetch": 1}, {"ctas_per_sm": 1, "kseg": 16},
                  {"stagger": 1, "kseg": 5}, {"stagger": 1, "prefetch": 0, "kseg": 1023},
                  {"kseg": 1023, "prefetch": 0, "ctas_per_sm": 2}):
        G.oras_tune(pc, **knobs)
        z = torch.empty_like(r)
        for _ in range(2):
            G.oras_apply(pc, r, z)
        G.oras_check_status(pc)
        assert (torch.linalg.norm(z - z0) / torch.linalg.norm(z0)).item() <= 1e-5, knobs
    best = G.oras_autotune(pc)
    assert 1 <= best["ctas_per_sm"] and 1 <= best["kseg"] <= 1023
    u = torch.zeros_like(r)
    res = G.cpm_gmres_solve(pc, r, u, tol=1e-8)[0]
    assert res["status"] == 0


@pytest.mark.parametrize("prec,tol", [("fp32", 1e-4), ("bf16", 3e-2)])
def test_tensor_core_lu_matches_cuda_core_lu(torus_uneven, prec, tol):
    # the tcgen05 trailing update (split-tf32 for FP32, bf16 inputs for BF16) factors the
    # same matrices as the CUDA-core update: M^{-1} r agrees to the factor precision
    band, part, oras, c = torus_uneven
    r = _dev(random_vector(oras.band.n_active, 17))
    out = []
    for simt in (False, True):
        pc = G.oras_setup(band, part, c, "oras", 4.0, 40.0, prec, simt_lu=simt)
        z = torch.empty_like(r)
        G.oras_apply(pc, r, z)
        G.oras_check_status(pc)
        out.append(z)
    err = (torch.linalg.norm(out[0] - out[1]) / torch.linalg.norm(out[1])).item()
    assert err <= tol, err
    ref = oras.M.apply(r.cpu().numpy())
    err_ref = np.linalg.norm(out[0].cpu().numpy() - ref) / np.linalg.norm(ref)
    assert err_ref <= (1e-3 if prec == "fp32" else 5e-2), err_ref


def test_algorithmic_band_preconditioner_and_solve():
    """The whole path on an algorithmic band (smallest interpolation-closed node set)."""
    from oracle import band as ob, geometry, interp, local, operator, partition, schwarz
    h, c, ns, no = 0.1, 1.0, 8, 2
    band = G.cpm_build_band("sphere", 1.0, 0.0, h, 3, construction="algorithmic")
    part = G.cpm_partition(band, ns, None, no)
    B = ob.build_band_algorithmic(geometry.Sphere(1.0), h, 3)
    E = interp.extension_matrix(B)
    A = operator.cpm_matrix(B, E, c)
    lab = partition.rcb(B.cp[:B.n_active], ns)
    marks = partition.CrossMarks(B, partition.cross_point_nodes(B, lab), no)
    lps = [local.oras_local(B, partition.build_subdomain(B, E, lab, j, no, True), c, 4.0, 40.0, marks)
           for j in range(ns)]
    M = schwarz.Schwarz(lps, B.n_active)
    pc = G.oras_setup(band, part, c, "oras", 4.0, 40.0, "fp64")
    r = random_vector(pc.n_active, 41)
    z = torch.empty(pc.n_active, dtype=torch.float64, device="cuda")
    G.oras_apply(pc, _dev(r), z)
    ref = M.apply(r)
    assert np.linalg.norm(z.cpu().numpy() - ref) / np.linalg.norm(ref) <= 1e-10
    cp = B.cp[:B.n_active]
    f = (c + 12.0) * cp[:, 0] * cp[:, 1] * cp[:, 2]
    u = torch.zeros(pc.n_active, dtype=torch.float64, device="cuda")
    res = G.cpm_gmres_solve(pc, _dev(f), u, tol=1e-12)[0]
    gref = krylov.fgmres(lambda x: A @ x, M.apply, f, 1e-12)
    assert res["status"] == 0 and abs(res["iterations"] - gref.iterations) <= 1
    assert np.linalg.norm(u.cpu().numpy() - gref.x) / np.linalg.norm(gref.x) <= 1e-10


@pytest.mark.gpu
def test_graph_partition_preconditioner_and_solve():
    """The graph bisection's subdomains (connected parts with irregular interfaces and more
    cross points than the coordinate cuts): M^{-1} r against the oracle built from the same
    labels (FP64 1e-10, FP32 1e-3) and the FGMRES solution."""
    h, c = 0.1, 1.0
    band = G.cpm_build_band("sphere", 1.0, 0.0, h, 3)
    part = G.cpm_partition(band, 8, None, 2, split="graph")
    P = problems.setup("sphere", 1.0, 0.0, h, 3, c, 8, 2, "oras", 4.0, 40.0, split="graph")
    assert np.array_equal(part.labels(), P.labels)
    r = random_vector(band.sizes()[0], 9)
    ref = P.M.apply(r)
    for prec, tol in (("fp64", 1e-10), ("fp32", 1e-3)):
        pc = G.oras_setup(band, part, c, "oras", 4.0, 40.0, prec)
        z = torch.empty(pc.n_active, dtype=torch.float64, device="cuda")
        G.oras_apply(pc, _dev(r), z)
        G.oras_check_status(pc)
        err = np.linalg.norm(z.cpu().numpy() - ref) / np.linalg.norm(ref)
        assert err <= tol, (prec, err)
    pc = G.oras_setup(band, part, c, "oras", 4.0, 40.0, "fp64")
    cp = band.info()["cp"][: pc.n_active]
    f = (c + 12.0) * cp[:, 0] * cp[:, 1] * cp[:, 2]
    u = torch.zeros(pc.n_active, dtype=torch.float64, device="cuda")
    res = G.cpm_gmres_solve(pc, _dev(f), u, tol=1e-12)[0]
    x = problems.solve(P, f, 1e-12).x
    assert res["status"] == 0
    assert np.linalg.norm(u.cpu().numpy() - x) <= 1e-10 * np.linalg.norm(x)
