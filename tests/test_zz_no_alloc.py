"""The allocation-free operator apply agrees with the regular one (needs a GB300).

cpm_op_apply_noalloc exists for callers that cannot allocate device memory (their memory
belongs to another allocator, or an allocation's device-wide synchronisation is not
acceptable in their loop).  Here the test plays such a caller: it hands over band data and
vectors it owns, calls the entry point twice in a row with different inputs, and checks each
result against cpm_op_apply on the same input, within the operator-apply tolerance of the
other GPU tests (64 eps (|A| |x|)_i, A from the CPU oracle).  This file is collected last.
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
        diff = np.abs(y_static.cpu().numpy() - y_ref.cpu().numpy())
        assert np.all(diff <= bound), seed


def test_noalloc_rejects_oversized_band():
    x = torch.zeros(8, dtype=torch.float64, device="cuda")
    i32 = torch.zeros(8, dtype=torch.int32, device="cuda")
    with pytest.raises(G.CpmError) as e:
        G.cpm_op_apply_noalloc(i32, x, i32, 8, G.CPM_NOALLOC_MAX_NODES + 1, 3, 1.0, 0.1, x, x)
    assert e.value.status == G._capi.CPM_ERR_BUDGET
