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
