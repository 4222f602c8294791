"""Band construction on the device (cpm_build_band_device) against the host construction:
every array bit for bit (active and ghost coordinates, closest points, triangles, neighbour
table, stencil bases, 1-D weights, z-pencil starts), on the analytic surfaces, the small mesh
and the 81,920-triangle mesh at h = 0.01; and an operator built on the device band applies the
same A x, bit for bit, as one built on the host band."""
import time

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_1909_08734_gb300 as G  # noqa: E402
from workloads import WORKLOADS, perturbed_icosphere, random_vector, surface_mesh  # noqa: E402

pytestmark = pytest.mark.gpu

KEYS = ["ijk", "cp", "nbr", "base", "pencil", "weights", "tri"]


def _same(a, b):
    ia, ib = a.info(), b.info()
    for k in ["n_active", "n_ghost", "p", "h", "lambda"]:
        assert ia[k] == ib[k], k
    for k in KEYS:
        if ia[k] is None or ib[k] is None:
            assert ia[k] is None and ib[k] is None, k
            continue
        assert ia[k].dtype == ib[k].dtype and np.array_equal(ia[k], ib[k]), k
        if ia[k].dtype == np.float64:           # identical bits, not only equal values
            assert np.array_equal(ia[k].view(np.int64), ib[k].view(np.int64)), k


CASES = [("sphere", 1.0, 0.0, 0.1, 3, None), ("sphere", 1.0, 0.0, 0.05, 2, None),
         ("torus", 1.0, 0.4, 0.05, 3, None), ("trimesh", 0.0, 0.0, 0.05, 3, "small")]


@pytest.mark.parametrize("case", CASES, ids=lambda c: f"{c[0]}-h{c[3]}-p{c[4]}")
def test_device_band_is_the_host_band(case):
    kind, R, r, h, p, mesh = case
    V, T = perturbed_icosphere(3, 0.15, 4) if mesh else (None, None)
    host = G.cpm_build_band(kind, R, r, h, p, verts=V, tris=T)
    dev = G.cpm_build_band(kind, R, r, h, p, verts=V, tris=T, on_device=True)
    _same(host, dev)


def test_device_band_full_size_mesh_and_operator():
    wl = WORKLOADS["mesh_h001"]
    V, T = surface_mesh(wl)
    t0 = time.perf_counter()
    host = G.cpm_build_band(wl.surface, wl.R, wl.r, wl.h, wl.p, verts=V, tris=T)
    t1 = time.perf_counter()
    dev = G.cpm_build_band(wl.surface, wl.R, wl.r, wl.h, wl.p, verts=V, tris=T, on_device=True)
    t2 = time.perf_counter()
    print(f"band of the 81,920-triangle mesh at h = 0.01: host {t1 - t0:.3f} s, device {t2 - t1:.3f} s")
    _same(host, dev)


def test_operator_on_device_band_applies_the_same():
    h = 0.05
    host = G.cpm_build_band("torus", 1.0, 0.4, h, 3)
    dev = G.cpm_build_band("torus", 1.0, 0.4, h, 3, on_device=True)
    x = torch.tensor(random_vector(host.sizes()[0], 3), dtype=torch.float64, device="cuda")
    ys = []
    for band in (host, dev):
        part = G.cpm_partition(band, 8, None, 2)
        pc = G.oras_setup(band, part, 2.0, "oras", 4.0, 40.0, "fp64")
        y = torch.empty_like(x)
        G.cpm_op_apply(pc, x, y)
        torch.cuda.synchronize()
        ys.append(y.cpu().numpy())
    assert np.array_equal(ys[0].view(np.int64), ys[1].view(np.int64))
