"""(O)RAS as a stationary solver (Eq. algRAS) through the C ABI against the oracle (GB300).

u_{k+1} = u_k + M^{-1}(f - A u_k), u_0 = 0.  With FP64 factors every iterate agrees with
the oracle's to the local solves' rounding (cond(A_j) eps per step, bound 1e-10 relative), so
the iteration counts agree exactly unless a residual lands within that rounding of the
threshold.  With FP32 / BF16 factors the FP64 residual makes the iteration converge to the
same fixed point (iterative refinement), only in more steps.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
import paper_1909_08734_gb300 as G  # noqa: E402
from oracle import problems, schwarz  # noqa: E402

pytestmark = pytest.mark.gpu


def _dev(x):
    return torch.tensor(np.ascontiguousarray(x), dtype=torch.float64, device="cuda")


@pytest.fixture(scope="module")
def sphere():
    h, c, ns, no = 0.1, 1.0, 8, 2
    band = G.cpm_build_band("sphere", 1.0, 0.0, h, 3)
    part = G.cpm_partition(band, ns, None, no)
    probs = {m: problems.setup("sphere", 1.0, 0.0, h, 3, c, ns, no, m, 4.0, 40.0) for m in ("ras", "oras")}
    cp = band.info()["cp"][: band.info()["n_active"]]
    f = (c + 12.0) * cp[:, 0] * cp[:, 1] * cp[:, 2]
    return band, part, probs, c, f


@pytest.mark.parametrize("method", ["ras", "oras"])
def test_stationary_fp64_matches_oracle(sphere, method):
    band, part, probs, c, f = sphere
    P = probs[method]
    pc = G.oras_setup(band, part, c, method, 4.0, 40.0, "fp64")
    u = torch.empty(pc.n_active, dtype=torch.float64, device="cuda")
    res = G.oras_stationary_solve(pc, _dev(f), u, tol=1e-8, max_it=400)[0]
    ref_u, ref_it, ok = schwarz.stationary_solve(P.A, P.M, f, 1e-8, 400)
    assert ok and res["status"] == 0
    assert res["iterations"] == ref_it
    U = u.cpu().numpy()
    assert np.linalg.norm(U - ref_u) / np.linalg.norm(ref_u) <= 1e-10
    true = np.linalg.norm(f - P.A @ U) / np.linalg.norm(f)
    assert abs(true - res["relres"]) <= 1e-12 and true <= 1e-8


def test_stationary_kth_iterate_matches_oracle(sphere):
    """Stopped after k steps (not converged): the k-th iterate equals the oracle's."""
    band, part, probs, c, f = sphere
    P = probs["oras"]
    pc = G.oras_setup(band, part, c, "oras", 4.0, 40.0, "fp64")
    u = torch.empty(pc.n_active, dtype=torch.float64, device="cuda")
    res = G.oras_stationary_solve(pc, _dev(f), u, tol=1e-14, max_it=3, raise_on_failure=False)[0]
    assert res["status"] == G._capi.CPM_ERR_NOT_CONVERGED and res["iterations"] == 3
    ref_u, it, ok = schwarz.stationary_solve(P.A, P.M, f, 1e-14, 3)
    assert not ok and it == 3
    assert np.linalg.norm(u.cpu().numpy() - ref_u) / np.linalg.norm(ref_u) <= 1e-11


def test_optimized_transmission_converges_faster(sphere):
    """Robin transmission conditions cut the stationary iteration count (Sec. 4)."""
    band, part, probs, c, f = sphere
    its = {}
    for method in ("ras", "oras"):
        pc = G.oras_setup(band, part, c, method, 4.0, 40.0, "fp64")
        u = torch.empty(pc.n_active, dtype=torch.float64, device="cuda")
        its[method] = G.oras_stationary_solve(pc, _dev(f), u, tol=1e-6, max_it=400)[0]["iterations"]
    assert its["oras"] < its["ras"], its


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_stationary_low_precision_reaches_fp64_fixed_point(sphere, prec):
    band, part, probs, c, f = sphere
    P = probs["oras"]
    pc = G.oras_setup(band, part, c, "oras", 4.0, 40.0, prec)
    u = torch.empty(pc.n_active, dtype=torch.float64, device="cuda")
    res = G.oras_stationary_solve(pc, _dev(f), u, tol=1e-10, max_it=800)[0]
    assert res["status"] == 0
    U = u.cpu().numpy()
    assert np.linalg.norm(f - P.A @ U) / np.linalg.norm(f) <= 1e-10 * (1 + 1e-3)


def test_stationary_zero_and_multi_rhs(sphere):
    band, part, probs, c, f = sphere
    pc = G.oras_setup(band, part, c, "oras", 4.0, 40.0, "fp64")
    n = pc.n_active
    F = np.stack([np.zeros(n), f, 2.0 * f])
    u = torch.full((3 * n,), 7.0, dtype=torch.float64, device="cuda")
    res = G.oras_stationary_solve(pc, _dev(F.ravel()), u, nrhs=3, tol=1e-9, max_it=400)
    assert [r["status"] for r in res] == [0, 0, 0]
    assert res[0]["iterations"] == 0 and res[0]["relres"] == 0.0
    U = u.cpu().numpy().reshape(3, n)
    assert np.all(U[0] == 0.0)
    assert res[1]["iterations"] == res[2]["iterations"]
    assert np.linalg.norm(U[2] - 2.0 * U[1]) <= 1e-12 * np.linalg.norm(U[2])
