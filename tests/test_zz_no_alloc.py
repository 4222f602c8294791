"""The allocation-free operator apply agrees with the regular one (needs a GB300).

cpm_op_apply_noalloc exists for callers that cannot allocate device memory (their memory
belongs to another allocator, or an allocation's device-wide synchronisation is not
acceptable in their loop).  Here the test plays such a caller: it hands over band data and
vectors it owns, calls the entry point twice in a row with different inputs, and checks each
result entry by entry against the CPU oracle's A x and against cpm_op_apply on the same input,
within the operator-apply tolerance of the other GPU tests (64 eps (|A| |x|)_i).  Arguments
of the wrong size or on another device are refused before any launch.  This file is
collected last.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
import paper_1909_08734_gb300 as G  # noqa: E402
from oracle import problems  # noqa: E402
from workloads import random_vector  # noqa: E402

pytestmark = pytest.mark.gpu
EPS = np.finfo(float).eps


def test_noalloc_apply_matches_regular_apply_twice():
    h, c = 0.1, 1.0
    band = G.cpm_build_band("sphere", 1.0, 0.0, h, 3)
    part = G.cpm_partition(band, 8, None, 2)
    pc = G.oras_setup(band, part, c, "ras", 0.0, 0.0, "fp64")
    info = band.info()
    n_a, n = info["n_active"], info["n_active"] + info["n_ghost"]
    dev = "cuda"
    pencil = torch.tensor(info["pencil"].ravel(), dtype=torch.int32, device=dev)
    weights = torch.tensor(info["weights"].ravel(), dtype=torch.float64, device=dev)
    nbr = torch.tensor(info["nbr"].ravel(), dtype=torch.int32, device=dev)
    A = problems.setup("sphere", 1.0, 0.0, h, 3, c, 8, 2, "ras").A
    absA = abs(A)
    for seed in (21, 22):                      # two calls in a row share the static scratch
        xh = random_vector(n_a, seed)
        x = torch.tensor(xh, dtype=torch.float64, device=dev)
        y_static = torch.full_like(x, float("nan"))
        y_ref = torch.empty_like(x)
        G.cpm_op_apply_noalloc(pencil, weights, nbr, n_a, n, 3, c, h, x, y_static)
        G.cpm_op_apply(pc, x, y_ref)
        torch.cuda.synchronize()
        bound = 64 * EPS * (absA @ np.abs(xh))
        ys = y_static.cpu().numpy()
        assert np.all(np.abs(ys - A @ xh) <= bound), seed           # the oracle's operator
        assert np.all(np.abs(ys - y_ref.cpu().numpy()) <= bound), seed


def test_noalloc_rejects_short_arguments_before_any_launch():
    band = G.cpm_build_band("sphere", 1.0, 0.0, 0.2, 3)
    info = band.info()
    n_a, n = info["n_active"], info["n_active"] + info["n_ghost"]
    pencil = torch.tensor(info["pencil"].ravel(), dtype=torch.int32, device="cuda")
    weights = torch.tensor(info["weights"].ravel(), dtype=torch.float64, device="cuda")
    nbr = torch.tensor(info["nbr"].ravel(), dtype=torch.int32, device="cuda")
    x = torch.zeros(n_a, dtype=torch.float64, device="cuda")
    y = torch.zeros_like(x)
    args = [pencil, weights, nbr, n_a, n, 3, 1.0, 0.2, x, y]
    for k, short in ((0, pencil[:-1]), (1, weights[:-16]), (2, nbr[:-6]), (8, x[:-1]), (9, y[:-1])):
        bad = list(args)
        bad[k] = short
        with pytest.raises(ValueError):
            G.cpm_op_apply_noalloc(*bad)
    with pytest.raises(ValueError):                      # a degree the pencils were not built for
        G.cpm_op_apply_noalloc(pencil, weights, nbr, n_a, n, 4, 1.0, 0.2, x, y)


def test_noalloc_rejects_oversized_band():
    # the entry point itself (below the binding's size checks) refuses a band larger than its
    # static scratch, before touching any pointer
    import ctypes as C
    x = torch.zeros(8, dtype=torch.float64, device="cuda")
    i32 = torch.zeros(8, dtype=torch.int32, device="cuda")
    p = lambda t: C.c_void_p(t.data_ptr())  # noqa: E731
    st = G._capi.load().cpm_op_apply_noalloc(p(i32), p(x), p(i32), 8, G.CPM_NOALLOC_MAX_NODES + 1, 3, 1.0, 0.1,
                                             p(x), p(x), None)
    assert st == G._capi.CPM_ERR_BUDGET
