"""Discrete extension operator E (Sec. 2.1, Fig. 1; barycentric form of Berrut & Trefethen).

Row k of E interpolates active-node values at the point y = CP(x_k) with a degree-p
tensor-product Lagrange polynomial on the (p+1)^3 grid nodes around y.

Per axis (reading of the stencil placement, which the paper leaves to its references):
  s = y / h,  b = floor(s - (p - 1)/2),  t = s - b  in [ (p-1)/2, (p+1)/2 ),
  nodes b, b+1, ..., b+p  (p = 3: b = floor(s) - 1, the 4 nodes around y).
1-D weights, second barycentric form on equispaced nodes m = 0..p:
  beta_m = (-1)^m C(p, m),  l_m(t) = (beta_m / (t - m)) / sum_n beta_n / (t - n),
  and l_m = delta_{m, t} when t is exactly a node.
Row weight of node (b_x + a, b_y + b, b_z + c) is (l^x_a * l^y_b) * l^z_c (Fig. 1 caption).
"""
from __future__ import annotations

from math import comb

import numpy as np
import scipy.sparse as sp


class StencilError(RuntimeError):
    """An interpolation stencil leaves the node set it must lie in."""


def stencil_base(Y: np.ndarray, h: float, p: int):
    """Lowest stencil node (int64, (N,3)) and local offsets t (float, (N,3)) of points Y."""
    S = Y / h
    B = np.floor(S - (p - 1) / 2.0)
    T = S - B
    return B.astype(np.int64), T


def bary_weights_1d(t: np.ndarray, p: int) -> np.ndarray:
    """Lagrange weights l_m(t), m = 0..p, at offsets t (N,), barycentric second form."""
    t = np.asarray(t, dtype=np.float64)
    beta = np.array([(-1) ** m * comb(p, m) for m in range(p + 1)], dtype=np.float64)
    diff = t[:, None] - np.arange(p + 1, dtype=np.float64)[None, :]
    with np.errstate(divide="ignore", invalid="ignore"):
        q = beta[None, :] / diff
        s = q[:, 0].copy()
        for m in range(1, p + 1):          # left-to-right sum
            s = s + q[:, m]
        W = q / s[:, None]
    exact = diff == 0.0
    rows = exact.any(axis=1)
    W[rows] = exact[rows].astype(np.float64)
    return W


def point_weights(Y: np.ndarray, h: float, p: int):
    """Stencil base and the three 1-D weight vectors for interpolation at points Y."""
    B, T = stencil_base(Y, h, p)
    Wx = bary_weights_1d(T[:, 0], p)
    Wy = bary_weights_1d(T[:, 1], p)
    Wz = bary_weights_1d(T[:, 2], p)
    return B, Wx, Wy, Wz


def stencil_offsets(p: int) -> np.ndarray:
    """(p+1)^3 offsets (a, b, c) in the order a slowest, c fastest."""
    r = np.arange(p + 1)
    A, Bb, C = np.meshgrid(r, r, r, indexing="ij")
    return np.stack([A.ravel(), Bb.ravel(), C.ravel()], axis=1)


def tensor_weights(Wx, Wy, Wz) -> np.ndarray:
    """(N, (p+1)^3) products (wx_a * wy_b) * wz_c in stencil_offsets order."""
    n, P = Wx.shape
    return ((Wx[:, :, None, None] * Wy[:, None, :, None]) * Wz[:, None, None, :]).reshape(n, P ** 3)


def interpolation_rows(band, Y: np.ndarray):
    """Global active columns (N, (p+1)^3) and weights of interpolation at points Y.

    Raises StencilError if any stencil node is not an active node."""
    p = band.p
    B, Wx, Wy, Wz = point_weights(Y, band.h, p)
    off = stencil_offsets(p)
    IJK = (B[:, None, :] + off[None, :, :]).reshape(-1, 3)
    cols = band.lookup(IJK).reshape(len(Y), -1)
    if np.any(cols < 0) or np.any(cols >= band.n_active):
        raise StencilError("interpolation stencil leaves the active set")
    return cols, tensor_weights(Wx, Wy, Wz)


def extension_matrix(band) -> sp.csr_matrix:
    """E in R^{(N_A + N_G) x N_A}: rows interpolate at CP(x_k) for every band node."""
    cols, vals = interpolation_rows(band, band.cp)
    n = band.n_nodes
    P3 = cols.shape[1]
    rows = np.repeat(np.arange(n), P3)
    return sp.csr_matrix((vals.ravel(), (rows, cols.ravel())), shape=(n, band.n_active))
