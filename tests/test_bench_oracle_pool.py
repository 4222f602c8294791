"""The all-cores CPU baseline computes exactly the oracle's preconditioner.

bench.py's OraclePool spreads the oracle's local SuperLU solves over spawned processes; every
worker factors the oracle's own local matrices, so M^{-1} r must equal
oracle.schwarz.Schwarz.apply bit for bit, and FGMRES with it must give the oracle's iterates.
"""
import numpy as np

import bench
from oracle import krylov, problems
from workloads import random_vector


def test_pool_apply_is_the_oracle_apply():
    P = problems.setup("sphere", 1.0, 0.0, 0.2, 3, 1.0, 5, 2, "oras", 4.0, 40.0)
    pool = bench.OraclePool(P, 2)
    try:
        for seed in (1, 2):
            r = random_vector(P.band.n_active, seed)
            assert np.array_equal(pool.apply(r), P.M.apply(r))
        f = random_vector(P.band.n_active, 3)
        a = krylov.fgmres(lambda v: P.A @ v, pool.apply, f, 1e-10, 50, 200)
        b = problems.solve(P, f, 1e-10)
        assert a.iterations == b.iterations and np.array_equal(a.x, b.x)
    finally:
        pool.close()
