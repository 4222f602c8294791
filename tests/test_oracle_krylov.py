"""Pins for the oracle's FGMRES (CPU only): Krylov least-squares optimality and exactness."""
import numpy as np

from oracle import krylov


def _matrix(n, seed):
    rng = np.random.default_rng(seed)
    return np.eye(n) * 4.0 + rng.standard_normal((n, n)) / np.sqrt(n)


def test_iterates_minimise_residual_over_krylov_space():
    n = 40
    A = _matrix(n, 0)
    f = np.random.default_rng(1).standard_normal(n)
    for k in range(1, 7):
        res = krylov.fgmres(lambda x: A @ x, lambda v: v, f, 1e-30, restart=50, stop_after=k)
        K = np.stack([np.linalg.matrix_power(A, i) @ f for i in range(k)], 1)
        c, *_ = np.linalg.lstsq(A @ K, f, rcond=None)
        assert np.allclose(res.x, K @ c, atol=1e-10)


def test_right_preconditioned_iterate_minimises_over_preconditioned_space():
    n = 30
    A = _matrix(n, 2)
    Minv = np.linalg.inv(np.diag(np.diag(A)) + 0.1)
    f = np.random.default_rng(3).standard_normal(n)
    for k in (2, 4):
        res = krylov.fgmres(lambda x: A @ x, lambda v: Minv @ v, f, 1e-30, stop_after=k)
        AM = A @ Minv
        K = np.stack([np.linalg.matrix_power(AM, i) @ f for i in range(k)], 1)
        c, *_ = np.linalg.lstsq(AM @ K, f, rcond=None)
        assert np.allclose(res.x, Minv @ K @ c, atol=1e-10)


def test_converges_to_dense_solution_with_restarts():
    n = 60
    A = _matrix(n, 4)
    f = np.random.default_rng(5).standard_normal(n)
    res = krylov.fgmres(lambda x: A @ x, lambda v: v, f, 1e-12, restart=5, max_it=500)
    xs = np.linalg.solve(A, f)
    kappa = np.linalg.cond(A)
    assert res.converged and res.relres <= 1e-12
    assert np.linalg.norm(res.x - xs) <= 10 * kappa * 1e-12 * np.linalg.norm(xs)


def test_zero_rhs():
    A = _matrix(10, 6)
    res = krylov.fgmres(lambda x: A @ x, lambda v: v, np.zeros(10), 1e-8)
    assert res.converged and res.iterations == 0 and not res.x.any()


def test_happy_breakdown_solves_exactly():
    # f = e_0 is an eigenvector of a diagonal A: w = A v_0 = 2 v_0 exactly, ||w|| = 0 after the
    # Gram-Schmidt pass, and the least-squares solution is the exact one (x = e_0 / 2)
    A = np.diag([2.0, 3.0, 5.0])
    f = np.array([1.0, 0.0, 0.0])
    res = krylov.fgmres(lambda x: A @ x, lambda v: v, f, 1e-12)
    assert res.converged and not res.breakdown and res.iterations == 1
    assert np.array_equal(res.x, np.array([0.5, 0.0, 0.0]))


def test_singular_hessenberg_is_breakdown_with_first_columns_only():
    # zero operator: A z_0 = 0, rho = 0 at k = 0, nothing is updated
    f = np.array([3.0, -4.0])
    res = krylov.fgmres(lambda x: 0.0 * x, lambda v: v, f, 1e-8)
    assert res.breakdown and not res.converged and res.iterations == 1
    assert not res.x.any() and res.relres == 1.0
    # nilpotent A (A e_1 = e_0, A e_0 = 0), f = e_1: step 0 gives H = [0; 1] (rotation c = 0,
    # s = 1), step 1 gives a zero column, so rho = 0 at k = 1; the update uses column 0 only,
    # whose least-squares coefficient is g_0 = 0 after the rotation: x stays 0, relres 1
    N = np.array([[0.0, 1.0], [0.0, 0.0]])
    res = krylov.fgmres(lambda x: N @ x, lambda v: v, np.array([0.0, 1.0]), 1e-8)
    assert res.breakdown and res.iterations == 2
    assert np.isfinite(res.x).all() and not res.x.any() and res.relres == 1.0
    # a restart limit hit at the same step reports non-convergence, not breakdown
    res = krylov.fgmres(lambda x: 0.0 * x, lambda v: v, f, 1e-8, max_it=1)
    assert not res.breakdown and not res.converged and res.iterations == 1
