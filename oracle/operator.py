"""Stabilised CPM matrix A = c I - Lap_S^h on the active nodes (Eq. impLapBel, Sec. 2.2).

Lap_S^h = -(2d/h^2) I + (Lap^h + (2d/h^2) [I 0]) E with d = 3 and Lap^h the 7-point
Laplacian, rows on Sigma_A, columns on Sigma_A u Sigma_G.  The 7-point diagonal -6/h^2
cancels against +(6/h^2)[I 0], so row i of Lap^h + (6/h^2)[I 0] is (1/h^2) times the sum
over the 6 neighbours, and

    (A x)_i = (c + 6/h^2) x_i - (1/h^2) sum_{k in N6(i)} (E x)_k.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp


def neighbour_sum_matrix(band) -> sp.csr_matrix:
    """N6 in {0,1}^{N_A x (N_A+N_G)}: row i has a 1 in each of the 6 neighbour columns."""
    n_a = band.n_active
    rows = np.repeat(np.arange(n_a), 6)
    return sp.csr_matrix((np.ones(6 * n_a), (rows, band.nbr.ravel())),
                         shape=(n_a, band.n_nodes))


def cpm_matrix(band, E: sp.csr_matrix, c: float) -> sp.csr_matrix:
    h = band.h
    diag = c + 6.0 / (h * h)
    invh2 = 1.0 / (h * h)
    N6 = neighbour_sum_matrix(band)
    A = sp.identity(band.n_active, format="csr") * diag - (N6 @ E) * invh2
    return A.tocsr()


def apply(band, E, c: float, x: np.ndarray) -> np.ndarray:
    """Matrix-free form of the same operator: v = E x on all nodes, then the 6-sum."""
    h = band.h
    v = E @ x
    return (c + 6.0 / (h * h)) * x - (1.0 / (h * h)) * v[band.nbr].sum(axis=1)
