"""Pins of the oracle's solvers against the trends of the paper's iteration-count tables.

The paper's counts come from METIS partitions at h = 1/50 and finer, which this build does not
reproduce (recursive bisection stands in for METIS), so exact counts are not a pin; the
qualitative facts the tables show are, and a mistake in the Robin rows, the cross-point weight
or the Schwarz iteration breaks them.  Unit sphere, p = 2, h = 0.05, f = (c + 12) xyz at the
closest points, c = 1, residual reduction 1e6 (Sec. 6):

* Table 2 (two subdomains, N_O = 4): ORAS at its best Robin weight needs well under half the
  RAS solver iterations; the count rises again for a large weight (ORAS tends to RAS as
  alpha -> infinity); as a preconditioner for GMRES every method needs fewer iterations than
  as a solver, and ORAS no more than RAS.
* Table 7 (subdomain count, N_O = 4, alpha = 4, alpha^x = 40): every count grows with the
  number of subdomains (no coarse space), and ORAS beats RAS as a solver at each count.
"""
import functools

import pytest

from oracle import krylov, problems, schwarz

H = 0.05
TOL = 1e-6


@functools.lru_cache(maxsize=None)
def counts(n_sub: int, method: str, alpha: float = 0.0):
    """(stationary solver iterations, FGMRES iterations) for one configuration."""
    if method == "oras":
        P = problems.setup("sphere", 1.0, 0.0, H, 2, 1.0, n_sub, 4, "oras", alpha, 10.0 * alpha)
    else:
        P = problems.setup("sphere", 1.0, 0.0, H, 2, 1.0, n_sub, 4, "ras")
    cp = P.band.cp[: P.band.n_active]
    f = 13.0 * cp[:, 0] * cp[:, 1] * cp[:, 2]
    _, it_s, ok = schwarz.stationary_solve(P.A, P.M, f, TOL, 3000)
    assert ok
    g = krylov.fgmres(lambda x: P.A @ x, P.M.apply, f, TOL, 50, 2000)
    assert g.converged
    return it_s, g.iterations


def test_robin_weight_trends_of_table2():
    ras = counts(2, "ras")
    oras = {a: counts(2, "oras", a) for a in (1.0, 2.0, 16.0)}
    best = min(s for s, _ in oras.values())
    assert 2 * best < ras[0], (oras, ras)                     # optimised Robin weight pays off
    assert best < oras[16.0][0] <= ras[0], (oras, ras)        # large weight drifts back to RAS
    for s, g in list(oras.values()) + [ras]:
        assert g < s, (oras, ras)                             # preconditioner beats solver
    assert min(g for _, g in oras.values()) <= ras[1], (oras, ras)


@pytest.mark.parametrize("method", ["ras", "oras"])
def test_counts_grow_with_subdomains_as_in_table7(method):
    a = 4.0 if method == "oras" else 0.0
    c2, c8, c32 = (counts(n, method, a) for n in (2, 8, 32))
    assert c2[0] < c8[0] < c32[0], (c2, c8, c32)
    assert c2[1] < c8[1] < c32[1], (c2, c8, c32)


def test_oras_beats_ras_as_solver_at_each_subdomain_count():
    for n in (2, 8, 32):
        assert counts(n, "oras", 4.0)[0] < counts(n, "ras")[0], n
