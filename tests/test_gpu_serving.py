"""Serving loop on the GPU: HBM-budget admission, batching, determinism, chains (GB300).

* oras_plan bounds what oras_setup and the solves actually allocate;
* cpm_vec_axpby against the FP64 formula;
* a request's solutions are bit-identical served alone and inside a mix that forces
  batching with other requests and evictions of its operator;
* a request that cannot fit the budget fails with CPM_ERR_BUDGET, the rest are served;
* continuous batching: batches on different operators run at once in separate slots (own
  stream and host thread), their CUDA-event intervals overlap on the device, and each result
  is bit-identical to serving it alone;
* served solutions agree with the oracle's sparse direct solve (A from the paper's
  discretisation, Eq. impLapBel), and a backward-Euler chain with c = 1/dt agrees with the
  oracle's chain u_n = A^{-1}(c u_{n-1}) to the solve tolerance times cond(A).
"""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

torch = pytest.importorskip("torch")
import paper_1909_08734_gb300 as G  # noqa: E402
from paper_1909_08734_gb300 import _capi  # noqa: E402
from paper_1909_08734_gb300.serving import Request, Server, overlap_seconds, summarize  # noqa: E402
from oracle import band as ob  # noqa: E402
from oracle import geometry, interp, operator  # noqa: E402
from workloads import perturbed_icosphere, smooth_rhs  # noqa: E402

pytestmark = pytest.mark.gpu
MESH = perturbed_icosphere(3, 0.15, 4)


def _server(**kw):
    s = Server(keep_solutions=True, **kw)
    s.register_surface("sphere", "sphere", 1.0, 0.0)
    s.register_surface("torus", "torus", 1.0, 0.4)
    s.register_surface("mesh", "trimesh", verts=MESH[0], tris=MESH[1])
    return s


def _req(srv, rid, surface, h, c, nrhs, seed, arrival=0.0, chain=0):
    cp = srv.band(surface, h)[2]
    return Request(rid, arrival, surface, h, c, smooth_rhs(cp, seed, nrhs), chain)


@pytest.mark.parametrize("prec", ["fp64", "fp32", "bf16"])
def test_plan_bounds_allocation(prec):
    band = G.cpm_build_band("torus", 1.0, 0.4, 0.05, 3)
    part = G.cpm_partition(band, 16, None, 2)
    plan = G.oras_plan(band, part, "oras", prec, 50, 1)
    pc = G.oras_setup(band, part, 10.0, "oras", 4.0, 40.0, prec)
    G.oras_autotune(pc)
    f = torch.randn(pc.n_active, dtype=torch.float64, device="cuda")
    u = torch.zeros_like(f)
    G.cpm_gmres_solve(pc, f, u, tol=1e-8)
    y = torch.empty_like(f)
    G.cpm_op_apply(pc, f, y)
    inf = pc.info()
    assert inf["factor_bytes"] == plan["factor_bytes"]
    assert inf["peak_device_bytes"] <= max(plan["setup_peak_bytes"], plan["resident_bytes"])
    assert inf["device_bytes"] <= plan["resident_bytes"]
    # the bound is not loose by more than the per-allocation page allowance and band copies
    assert plan["resident_bytes"] <= 1.3 * inf["device_bytes"] + (256 << 20)


def test_vec_axpby():
    n = 100003
    g = torch.Generator(device="cpu").manual_seed(3)
    x = torch.randn(n, dtype=torch.float64, generator=g)
    y = torch.randn(n, dtype=torch.float64, generator=g)
    xd, yd = x.cuda(), y.cuda()
    G.cpm_vec_axpby(2.5, xd, 0.0, yd)
    assert torch.equal(yd.cpu(), 2.5 * x)
    yd = y.cuda()
    G.cpm_vec_axpby(-0.75, xd, 1.25, yd)
    ref = -0.75 * x.numpy() + 1.25 * y.numpy()
    bound = 2 * np.finfo(float).eps * (np.abs(0.75 * x.numpy()) + np.abs(1.25 * y.numpy()))
    assert np.all(np.abs(yd.cpu().numpy() - ref) <= bound)


def test_alone_and_mixed_results_are_bit_identical():
    probe = dict(surface="torus", h=0.05, c=3.0, nrhs=3, seed=11)
    a = _server(precision="fp32")
    alone = a.serve([_req(a, 0, **probe)])[0]
    a.close()
    assert alone.status == 0
    # mix: a budget that holds roughly one operator at a time; the probe's operator is set up,
    # evicted by other operators, set up again, and the probe is batched with another request
    b = _server(precision="fp32")
    band, part, _ = b.band("torus", 0.05)
    plan = G.oras_plan(band, part, "oras", "fp32", 50, 1)
    b.budget = int(1.6 * max(plan["setup_peak_bytes"], plan["resident_bytes"]))
    first = b.serve([_req(b, 2, "torus", 0.05, 3.0, 2, 7),
                     _req(b, 1, "sphere", 0.05, 1.0, 2, 5, arrival=0.001),
                     _req(b, 3, "mesh", 0.05, 0.5, 1, 9, arrival=0.002)], realtime=False)
    assert all(r.status == 0 for r in first)
    second = b.serve([_req(b, 0, **probe),
                      _req(b, 6, "torus", 0.05, 3.0, 2, 17),
                      _req(b, 4, "torus", 0.05, 3.0, 1, 13, arrival=0.001, chain=2),
                      _req(b, 5, "sphere", 0.05, 20.0, 4, 15, arrival=0.002)], realtime=False)
    out = {r.rid: r for r in second}
    assert all(r.status == 0 for r in out.values())
    assert b.counters["evictions"] >= 2
    mixed = out[0]
    assert mixed.factorised and mixed.batch_rhs == mixed.nrhs + 2   # re-set-up, batched with 6
    assert np.array_equal(mixed.u, alone.u)
    assert mixed.iterations == alone.iterations
    b.close()


def test_batches_on_different_operators_overlap_on_the_device():
    specs = [("sphere", 0.05, 1.0, 4, 41), ("torus", 0.05, 2.0, 4, 43), ("sphere", 0.05, 7.0, 2, 45)]
    alone = {}
    for k, sp in enumerate(specs):
        s = _server(precision="fp32", slots=1)
        alone[k] = s.serve([_req(s, k, *sp)], realtime=False)[0]
        s.close()
    s = _server(precision="fp32", slots=3)
    out = {r.rid: r for r in s.serve([_req(s, k, *sp) for k, sp in enumerate(specs)], realtime=False)}
    assert all(r.status == 0 for r in out.values())
    assert sorted(r.slot for r in out.values()) == [0, 1, 2]
    assert len(s.batches) == 3 and overlap_seconds(s.batches) > 0.0
    for k, r in out.items():
        assert np.array_equal(r.u, alone[k].u), k
        assert r.iterations == alone[k].iterations
    s.close()


def test_budget_rejection_and_admission():
    s = _server(precision="fp32")
    band, part, _ = s.band("sphere", 0.05)
    plan = G.oras_plan(band, part, "oras", "fp32", 50, 1)
    s.budget = int(1.2 * max(plan["setup_peak_bytes"], plan["resident_bytes"]))
    reqs = [_req(s, 0, "sphere", 0.05, 1.0, 1, 1),
            _req(s, 1, "torus", 0.025, 1.0, 1, 2),          # larger operator: cannot fit
            _req(s, 2, "sphere", 0.05, 2.0, 1, 3)]
    out = {r.rid: r for r in s.serve(reqs, realtime=False)}
    assert out[0].status == 0 and out[2].status == 0
    assert out[1].status == _capi.CPM_ERR_BUDGET
    st = summarize(list(out.values()))
    assert st["rejected_budget"] == 1 and st["served"] == 2
    s.close()


def _oracle_matrix(kind, R, r, h, c, V=None, T=None):
    B = ob.build_band(geometry.make_surface(kind, R, r, V, T), h, 3)
    return operator.cpm_matrix(B, interp.extension_matrix(B), c), B


@pytest.mark.parametrize("surface", ["sphere", "mesh"])
def test_served_solutions_match_direct_solve(surface):
    h, c = 0.1, 2.0
    s = _server(precision="fp32", tol=1e-10)
    r = s.serve([_req(s, 0, surface, h, c, 2, 21)], realtime=False)[0]
    assert r.status == 0 and max(r.relres) <= 1e-10
    kind, R, rr, V, T = ("sphere", 1.0, 0.0, None, None) if surface == "sphere" else \
        ("trimesh", 0.0, 0.0, MESH[0], MESH[1])
    A, B = _oracle_matrix(kind, R, rr, h, c, V, T)
    lu = spla.splu(A.tocsc())
    F = smooth_rhs(B.cp[:B.n_active], 21, 2)
    kappa = (c + 12 / h ** 2) / c
    for k in range(2):
        ref = lu.solve(F[k])
        assert np.linalg.norm(r.u[k] - ref) <= 2 * kappa * 1e-10 * np.linalg.norm(ref)
    s.close()


def test_backward_euler_chain_matches_oracle():
    # h = 0.05: the tube plus its ghost layer stays inside the torus' reach r = 0.4
    h, c, steps = 0.05, 50.0, 4                     # dt = 1/c
    s = _server(precision="fp32", tol=1e-11)
    r = s.serve([_req(s, 0, "torus", h, c, 1, 31, chain=steps)], realtime=False)[0]
    assert r.status == 0 and len(r.iterations) == steps + 1
    A, B = _oracle_matrix("torus", 1.0, 0.4, h, c)
    lu = spla.splu(A.tocsc())
    u = lu.solve(smooth_rhs(B.cp[:B.n_active], 31, 1)[0])
    for _ in range(steps):
        u = lu.solve(c * u)
    kappa = (c + 12 / h ** 2) / c
    assert np.linalg.norm(r.u[0] - u) <= 2 * (steps + 1) * kappa * 1e-11 * np.linalg.norm(u)
    s.close()
