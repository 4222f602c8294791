"""Local subdomain operators for RAS and ORAS (Sec. 2.2 Eq. simpleRAS; Sec. 5 Eq. localOP).

RAS (Dirichlet transmission): A_j = R_j A R_j^T on Sigma_j (Eq. simpleRAS), local
  unknowns = Sigma_j in global order.

ORAS (Robin transmission, Sec. 5.2): local unknowns = Sigma_j then Sigma_j^{BC,A}, each in
  global order (n_j = |Sigma_j| + |Sigma_j^{BC,A}|).  Eq. localOP,
      A_j = (c + 6/h^2) I - (6/h^2 + Lap_j^h) [E_j ; T_j],
  gives, for a row i with a full 7-point stencil,
      (A_j w)_i = (c + 6/h^2) w_i - (1/h^2) sum_{k in N6(i)} v_k(w),
  where v_k is the extension of w to node k:
      k in Sigma_j u Sigma_j^G : v_k = E-row of k (interpolation at CP_S(x_k)),
      k in Sigma_j^BC          : v_k = T-row of k = interpolation at CP_{S_j}(x_k)
                                 divided by (1 + alpha_k d_k . q_k)          (Eq. robfo).
  d_k = x_k - CP_{S_j}(x_k) (Sec. 4.2); with n the unit surface normal at CP_{S_j}(x_k),
  d_k . q_k = |d_k - (d_k . n) n| exactly when q_k follows Eq. naConorm, and is 0 (so the
  row is the plain extension) when d_k is parallel to n.
  alpha_k = alpha_x near cross points (Sec. 5.2.2), alpha elsewhere.

Reading R1 (default): every local unknown, including Sigma_j^{BC,A}, gets the row above;
  this is why Sec. 4.1 adds, for Robin conditions only, a ghost layer around the active
  boundary nodes (their 7-point stencils need it).
Reading R3 (option): rows of Sigma_j^{BC,A} are (c + 6/h^2) w_i - (6/h^2) (T w)_i, i.e.
  Lap_j^h has no rows there; no boundary ghost layer is used.
Right-hand side of every local problem: [R_j r ; 0] (Sec. 5, after Eq. localOP).
Parity status: the assembled rows are pinned against the mathematics for analytic surfaces
  (first-order convergence with exact Robin data under R1 and R3, the alpha -> infinity
  Dirichlet limit, tests/test_oracle_robin.py); the choice between R1 and R3 is a reading.
"""
from __future__ import annotations

import dataclasses

import numpy as np
import scipy.sparse as sp

from . import interp
from .geometry import norm3
from .partition import effective_boundary_cp


@dataclasses.dataclass
class LocalProblem:
    j: int
    unknowns: np.ndarray      # global active index of each local unknown
    n_sigma: int              # the first n_sigma unknowns are Sigma_j
    A: sp.csr_matrix
    own_local: np.ndarray     # local positions of the disjoint set
    own_global: np.ndarray    # their global indices
    # Robin boundary data (ORAS only): BC node, CP_{S_j}, generator, d.q, alpha
    bc_nodes: np.ndarray | None = None
    bc_cp: np.ndarray | None = None
    bc_gen: np.ndarray | None = None
    bc_dq: np.ndarray | None = None
    bc_alpha: np.ndarray | None = None

    @property
    def n(self) -> int:
        return len(self.unknowns)

    def rhs(self, r: np.ndarray) -> np.ndarray:
        """[R_j r ; 0]: residual on Sigma_j, zero on the boundary unknowns."""
        b = np.zeros(self.n)
        b[:self.n_sigma] = r[self.unknowns[:self.n_sigma]]
        return b


def _own_positions(sub, unknowns):
    pos = np.searchsorted(sub.sigma, sub.own)
    assert np.array_equal(sub.sigma[pos], sub.own)
    return pos


def ras_local(A: sp.csr_matrix, sub) -> LocalProblem:
    """A_j = R_j A R_j^T (Eq. simpleRAS)."""
    U = sub.sigma
    Aj = A[U][:, U].tocsr()
    return LocalProblem(sub.j, U, len(U), Aj, _own_positions(sub, U), sub.own)


def robin_rows(band, sub, nodes, near_cross, alpha: float, alpha_x: float):
    """T-rows of boundary nodes (Eq. locCP, Eq. naConorm, Eq. robfo).

    Returns global active columns (M, (p+1)^3), scaled weights, CP_{S_j}, generator tags,
    d.q and alpha per node."""
    y, gen = effective_boundary_cp(band, sub, nodes)
    cols, w = interp.interpolation_rows(band, y)
    X = band.coords(nodes)
    d = X - y
    nrm = band.node_normals(gen)                    # normal at CP_{S_j} = CP(generator)
    dn = (d[:, 0] * nrm[:, 0] + d[:, 1] * nrm[:, 1]) + d[:, 2] * nrm[:, 2]
    dperp = d - dn[:, None] * nrm
    dq = norm3(dperp)
    a = np.where(near_cross(nodes), alpha_x, alpha)
    scale = 1.0 / (1.0 + a * dq)
    return cols, w * scale[:, None], y, gen, dq, a


def oras_local(band, sub, c: float, alpha: float, alpha_x: float, near_cross,
               reading: str = "R1") -> LocalProblem:
    n_a = band.n_active
    h = band.h
    diag = c + 6.0 / (h * h)
    invh2 = 1.0 / (h * h)
    U = np.concatenate([sub.sigma, sub.bc_a])
    n, ns = len(U), len(sub.sigma)
    loc = np.full(n_a, -1, dtype=np.int64)
    loc[U] = np.arange(n)

    interior = np.concatenate([sub.sigma, sub.ghost])
    bc = np.concatenate([sub.bc_a, sub.bc_g]) if reading == "R1" else sub.bc_a
    cols_i, w_i = interp.interpolation_rows(band, band.cp[interior])
    if len(bc):
        cols_b, w_b, y, gen, dq, a = robin_rows(band, sub, bc, near_cross, alpha, alpha_x)
    else:
        P3 = (band.p + 1) ** 3
        cols_b, w_b = np.zeros((0, P3), np.int64), np.zeros((0, P3))
        y, gen, dq, a = np.zeros((0, 3)), np.zeros(0, np.int64), np.zeros(0), np.zeros(0)
    vcols = loc[np.concatenate([cols_i, cols_b])]
    if np.any(vcols < 0):
        raise interp.StencilError("local extension stencil leaves the local unknowns")
    vvals = np.concatenate([w_i, w_b])
    nodes = np.concatenate([interior, bc])
    pos = np.full(band.n_nodes, -1, dtype=np.int64)
    pos[nodes] = np.arange(len(nodes))

    n_pde = n if reading == "R1" else ns
    nb = pos[band.nbr[U[:n_pde]]]                       # (n_pde, 6)
    if np.any(nb < 0):
        raise interp.StencilError("7-point stencil of a local row leaves the local nodes")
    P3 = vcols.shape[1]
    rr = np.repeat(np.arange(n_pde), 6 * P3)
    cc = vcols[nb].reshape(-1)
    vv = (-invh2 * vvals[nb]).reshape(-1)
    parts_r = [rr, np.arange(n)]
    parts_c = [cc, np.arange(n)]
    parts_v = [vv, np.full(n, diag)]
    if reading == "R3" and n > ns:
        bpos = pos[U[ns:]]
        parts_r.append(np.repeat(np.arange(ns, n), P3))
        parts_c.append(vcols[bpos].reshape(-1))
        parts_v.append((-(6.0 * invh2) * vvals[bpos]).reshape(-1))
    Aj = sp.coo_matrix((np.concatenate(parts_v), (np.concatenate(parts_r), np.concatenate(parts_c))),
                       shape=(n, n)).tocsr()
    Aj.sum_duplicates()
    return LocalProblem(sub.j, U, ns, Aj, _own_positions(sub, U), sub.own,
                        bc, y, gen, dq, a)
