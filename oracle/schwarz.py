"""Restricted additive Schwarz preconditioner and solver (Sec. 2.2, Eqs. restCons, algRAS).

M^{-1} r = sum_j  Rtilde_j^T (A_j^{-1} [R_j r ; 0])|_{disjoint set of j}
Each global unknown belongs to exactly one disjoint set, so the restricted prolongation
writes every entry of z once.  Local solves use LU factorisations (Sec. 5): SciPy's sparse
SuperLU, or dense partial-pivoting LU for small cross-checks.
Stationary (O)RAS solver: u <- u + M^{-1}(f - A u)  (Eq. algRAS).
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla
import scipy.sparse.linalg as spla


class Schwarz:
    def __init__(self, local_problems, n_active: int, dense: bool = False):
        self.lps = local_problems
        self.n_active = n_active
        self.dense = dense
        self.factors = []
        for lp in local_problems:
            if dense:
                self.factors.append(sla.lu_factor(lp.A.toarray()))
            else:
                self.factors.append(spla.splu(lp.A.tocsc()))

    def local_solve(self, j: int, b: np.ndarray) -> np.ndarray:
        f = self.factors[j]
        return sla.lu_solve(f, b) if self.dense else f.solve(b)

    def apply(self, r: np.ndarray) -> np.ndarray:
        z = np.zeros(self.n_active)
        for j, lp in enumerate(self.lps):
            e = self.local_solve(j, lp.rhs(r))
            z[lp.own_global] = e[lp.own_local]
        return z


def stationary_solve(A, M: Schwarz, f: np.ndarray, tol: float, max_it: int):
    """(O)RAS as a solver; stops when ||f - A u|| <= tol ||f||."""
    u = np.zeros_like(f)
    nf = np.linalg.norm(f)
    r = f.copy()
    for it in range(1, max_it + 1):
        u = u + M.apply(r)
        r = f - A @ u
        if np.linalg.norm(r) <= tol * nf:
            return u, it, True
    return u, max_it, False
