"""Failure detection on the GPU without a GPU fault (needs a GB300).

* A bounded device wait is made to expire (an mbarrier phase and a flag that nothing
  completes): the kernel returns, the handle's status reports CPM_ERR_TIMEOUT once, and the
  same context then solves normally.
* A NaN in the right-hand side is reported as CPM_ERR_NAN by FGMRES and by the stationary
  solver, and the next solve on the same handle succeeds.
* A zero pivot (one local column zeroed by the set-up self-test) is reported as
  CPM_ERR_SINGULAR with the subdomain it belongs to.
* A singular Hessenberg matrix (the operator made the zero matrix by a self-test, so that
  A z_0 = 0 while the residual is still ||f||) is reported as CPM_ERR_BREAKDOWN after one
  iteration with u unchanged, on its own and next to a zero right-hand side in a lock-step
  batch, with and without the captured iteration graph.
"""
import time

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import paper_1909_08734_gb300 as G  # noqa: E402
from paper_1909_08734_gb300 import _capi  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pc():
    band = G.cpm_build_band("sphere", 1.0, 0.0, 0.1, 3)
    part = G.cpm_partition(band, 8, None, 2)
    return G.oras_setup(band, part, 1.0, "oras", 4.0, 40.0, "fp32")


def _f(pc):
    cp = pc.band.info()["cp"][: pc.n_active]
    return torch.tensor(13.0 * cp[:, 0] * cp[:, 1] * cp[:, 2], dtype=torch.float64, device="cuda")


def test_expired_wait_is_reported_and_context_survives(pc):
    t0 = time.time()
    st = G.cpm_selftest_bounded_wait(pc, 0.2)
    dt = time.time() - t0
    assert st == _capi.CPM_ERR_TIMEOUT
    assert 0.2 <= dt < 10.0
    with pytest.raises(G.CpmError) as e:
        G.oras_check_status(pc)
    assert e.value.status == _capi.CPM_ERR_TIMEOUT
    G.oras_check_status(pc)                       # reported once, then cleared
    f = _f(pc)
    u = torch.zeros_like(f)
    res = G.cpm_gmres_solve(pc, f, u, tol=1e-8)[0]
    assert res["status"] == 0 and res["relres"] <= 1e-8


def test_nan_rhs_is_reported(pc):
    f = _f(pc)
    bad = f.clone()
    bad[17] = float("nan")
    u = torch.zeros_like(f)
    res = G.cpm_gmres_solve(pc, bad, u, tol=1e-8, raise_on_failure=False)[0]
    assert res["status"] == _capi.CPM_ERR_NAN
    res = G.oras_stationary_solve(pc, bad, u, tol=1e-8, max_it=10, raise_on_failure=False)[0]
    assert res["status"] == _capi.CPM_ERR_NAN
    with pytest.raises(G.CpmError) as e:
        G.cpm_gmres_solve(pc, bad, u, tol=1e-8)
    assert e.value.status == _capi.CPM_ERR_NAN
    res = G.cpm_gmres_solve(pc, f, u, tol=1e-8)[0]
    assert res["status"] == 0 and np.isfinite(u.cpu().numpy()).all()


@pytest.mark.parametrize("prec", ["fp64", "fp32", "bf16"])
def test_zero_pivot_is_reported_with_its_subdomain(prec):
    # valid inputs (c > 0) give nonsingular local matrices, so the self-test zeroes one local
    # column of subdomain 2 between assembly and factorisation; the factorisation must report
    # CPM_ERR_SINGULAR naming that subdomain, and the band then sets up normally
    band = G.cpm_build_band("sphere", 1.0, 0.0, 0.2, 3)
    part = G.cpm_partition(band, 4, None, 2)
    st, msg = G.oras_setup_selftest_singular(band, part, 1.0, "oras", 4.0, 40.0, prec, 2)
    assert st == _capi.CPM_ERR_SINGULAR, (st, msg)
    assert "subdomain 2" in msg, msg
    pc = G.oras_setup(band, part, 1.0, "oras", 4.0, 40.0, prec)
    f = _f(pc)
    u = torch.zeros_like(f)
    assert G.cpm_gmres_solve(pc, f, u, tol=1e-8)[0]["status"] == 0


@pytest.mark.parametrize("nrhs,use_graph,zero_second", [(1, True, False), (1, False, False), (2, True, True),
                                                         (2, False, False)])
def test_singular_hessenberg_is_reported_as_breakdown(nrhs, use_graph, zero_second):
    band = G.cpm_build_band("sphere", 1.0, 0.0, 0.1, 3)
    part = G.cpm_partition(band, 8, None, 2)
    pc = G.oras_setup(band, part, 1.0, "oras", 4.0, 40.0, "fp32")
    f1 = _f(pc)
    x = torch.linspace(-1.0, 1.0, pc.n_active, dtype=torch.float64, device="cuda")
    y = torch.empty_like(x)
    G.cpm_op_apply(pc, x, y)
    assert torch.count_nonzero(y).item() > 0
    G.cpm_selftest_zero_operator(pc)
    G.cpm_op_apply(pc, x, y)
    assert torch.count_nonzero(y).item() == 0     # A = 0 exactly
    rows = [f1] + [torch.zeros_like(f1) if zero_second else 2.0 * f1][: nrhs - 1]
    f = torch.cat(rows).contiguous()
    u = torch.zeros_like(f)
    res = G.cpm_gmres_solve(pc, f, u, nrhs=nrhs, tol=1e-8, use_graph=use_graph, raise_on_failure=False)
    for q, r in enumerate(res):
        if q == 1 and zero_second:                # ||f|| = 0: converged before the first step
            assert r["status"] == 0 and r["iterations"] == 0, r
            continue
        assert r["status"] == _capi.CPM_ERR_BREAKDOWN, r
        assert r["iterations"] == 1, r
        assert abs(r["relres"] - 1.0) < 1e-14, r  # nothing was updated: r = f
    assert torch.count_nonzero(u).item() == 0
    with pytest.raises(G.CpmError) as e:
        G.cpm_gmres_solve(pc, f, u, nrhs=nrhs, tol=1e-8, use_graph=use_graph)
    assert e.value.status == _capi.CPM_ERR_BREAKDOWN
