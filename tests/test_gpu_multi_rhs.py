"""Several right-hand sides per streamed factor tile (needs a GB300).

One launch of the batched solve applies M^{-1} to up to 8 right-hand sides, each column
through exactly the same operations as a single right-hand side, so the results are
bit-identical to one-at-a-time applications; the stationary solver iterates several
right-hand sides together with the same guarantee.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
import paper_1909_08734_gb300 as G  # noqa: E402
from workloads import random_vector  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def bp():
    band = G.cpm_build_band("torus", 1.0, 0.4, 0.05, 3)
    part = G.cpm_partition(band, 16, None, 2)
    return band, part


@pytest.mark.parametrize("prec", ["fp64", "fp32", "bf16"])
@pytest.mark.parametrize("nrhs", [3, 8, 11])
def test_multi_rhs_apply_is_bitwise_single_rhs(bp, prec, nrhs):
    band, part = bp
    pc = G.oras_setup(band, part, 10.0, "oras", 4.0, 40.0, prec)
    n = pc.n_active
    R = torch.tensor(np.stack([random_vector(n, 100 + q) for q in range(nrhs)]), dtype=torch.float64,
                     device="cuda")
    Z = torch.empty_like(R)
    G.oras_apply(pc, R.view(-1), Z.view(-1), nrhs=nrhs)
    G.oras_check_status(pc)
    for q in range(nrhs):
        z = torch.empty(n, dtype=torch.float64, device="cuda")
        G.oras_apply(pc, R[q].contiguous(), z)
        assert torch.equal(z, Z[q]), q
    # a solve afterwards recaptures its graph with the grown buffers
    f = R[0].contiguous()
    u = torch.zeros_like(f)
    res = G.cpm_gmres_solve(pc, f, u, tol=1e-8)[0]
    assert res["status"] == 0


def test_multi_rhs_stationary_is_bitwise_single_rhs(bp):
    band, part = bp
    pc = G.oras_setup(band, part, 10.0, "oras", 4.0, 40.0, "fp32")
    n = pc.n_active
    F = np.stack([random_vector(n, 200 + q) for q in range(5)])
    F[2] *= 0.0                                     # a zero right-hand side in the batch
    Fd = torch.tensor(F, dtype=torch.float64, device="cuda")
    U = torch.empty_like(Fd)
    res = G.oras_stationary_solve(pc, Fd.view(-1), U.view(-1), nrhs=5, tol=1e-8, max_it=500)
    assert [r["status"] for r in res] == [0] * 5 and res[2]["iterations"] == 0
    for q in range(5):
        u = torch.empty(n, dtype=torch.float64, device="cuda")
        r1 = G.oras_stationary_solve(pc, Fd[q].contiguous(), u, tol=1e-8, max_it=500)[0]
        assert r1["iterations"] == res[q]["iterations"]
        assert torch.equal(u, U[q]), q


@pytest.mark.parametrize("prec", ["fp64", "fp32", "bf16"])
@pytest.mark.parametrize("nrhs,restart,use_graph", [(3, 50, True), (8, 6, True), (5, 6, False)])
def test_lock_step_gmres_is_bitwise_single_rhs(bp, prec, nrhs, restart, use_graph):
    # FGMRES over several right-hand sides in lock step (one solve launch per iteration for
    # all of them) gives every right-hand side exactly its single-rhs iterates: the same
    # iteration count, residual and solution bits, also when right-hand sides stop in
    # different restart cycles (restart 6) and with a zero right-hand side in the batch.
    band, part = bp
    pc = G.oras_setup(band, part, 10.0, "oras", 4.0, 40.0, prec)
    n = pc.n_active
    F = np.stack([random_vector(n, 300 + q) * (1.0 + 3.0 * q) for q in range(nrhs)])
    F[1] *= 0.0
    if nrhs > 2:
        F[2] = F[0] + 1e-3 * F[2]                   # a near-duplicate converging at a similar step
    Fd = torch.tensor(F, dtype=torch.float64, device="cuda")
    U = torch.zeros_like(Fd)
    res = G.cpm_gmres_solve(pc, Fd.view(-1), U.view(-1), nrhs=nrhs, tol=1e-9, restart=restart,
                            max_it=600, use_graph=use_graph)
    assert all(r["status"] == 0 for r in res), res
    assert res[1]["iterations"] == 0 and torch.count_nonzero(U[1]).item() == 0
    for q in range(nrhs):
        u = torch.zeros(n, dtype=torch.float64, device="cuda")
        r1 = G.cpm_gmres_solve(pc, Fd[q].contiguous(), u, tol=1e-9, restart=restart, max_it=600,
                               use_graph=use_graph)[0]
        assert r1["iterations"] == res[q]["iterations"], (q, r1, res[q])
        assert r1["relres"] == res[q]["relres"], q
        assert torch.equal(u, U[q]), q
