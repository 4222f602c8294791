"""Disjoint and overlapping subdomains and their node sets (Secs. 3, 4.1, 4.2, 5.2.2).

Disjoint split (replaces METIS, Sec. 3.1): recursive coordinate bisection of the closest
points of Sigma_A.  At a bisection-tree node holding n points and leaves [l0, l1):
  axis = the coordinate of largest extent of the points' CP bounding box (ties: x < y < z);
  points ordered by (CP[axis], global index);
  left leaves [l0, l0 + P//2), n_left = floor(n * W_left / W) with integer leaf weights.
Graph split (also standing in for METIS's partition of the nearest-neighbour graph,
  Sec. 3.1): recursive bisection of the active 6-neighbour graph by the difference of the
  graph distances to two pseudo-peripheral nodes, then size-keeping swap passes
  (graph_bisection); the same leaf rule.
Interface alignment (Sec. 3.2), optional passes after the split: an interface node (an
  active node with an active 6-neighbour of another label) whose nearest grid point to its
  closest point, round(CP/h) = floor(CP/h + 0.5) per axis, carries another label moves to
  that label; all moves of a pass are decided on the labels before the pass.
Overlap (Sec. 4.1): Sigma_j = active nodes within N_O steps of the disjoint set in the
  6-neighbour graph on Sigma_A; the last layer is BFS distance exactly N_O.
Sigma_j^G (Sec. 4.1): ghost nodes among the 6-neighbours of Sigma_j.
Sigma_j^BC (Sec. 4.1): active nodes completing the 7-point stencils of Sigma_j and the
  interpolation stencils of CP(x), x in Sigma_j u Sigma_j^G, that are not in Sigma_j;
  for Robin conditions also the ghost layer N6(Sigma_j^{BC,A}) \\ (everything above).
Lambda_j (Sec. 4.2): CP(x) for x in the last overlap layer, tagged by x's global index.
CP_{S_j}(x_i) (Eq. locCP): the point of Lambda_j nearest to x_i (ties: lowest tag).
Cross-point nodes (Sec. 5.2.2 of the method, "Modified scheme for cross points"): active
  nodes whose active 6-neighbours carry >= 2 labels other than their own; BC nodes within
  2 N_O h of any of them (squared integer grid distance <= (2 N_O)^2) use alpha_x.
"""
from __future__ import annotations

import collections
import dataclasses

import numpy as np

from .band import NBR_OFFSETS


def rcb(points: np.ndarray, n_sub: int, leaf_weights=None) -> np.ndarray:
    """Labels in [0, n_sub) for each point (recursive coordinate bisection)."""
    n = len(points)
    w = np.ones(n_sub, dtype=np.int64) if leaf_weights is None else np.asarray(leaf_weights, np.int64)
    labels = np.full(n, -1, dtype=np.int64)
    stack = [(np.arange(n, dtype=np.int64), 0, n_sub)]
    while stack:
        idx, l0, l1 = stack.pop()
        P = l1 - l0
        if P == 1:
            labels[idx] = l0
            continue
        pts = points[idx]
        ext = pts.max(axis=0) - pts.min(axis=0)
        axis = int(np.argmax(ext))                 # first maximum: x < y < z
        order = np.lexsort((idx, pts[:, axis]))    # primary CP[axis], secondary index
        sidx = idx[order]
        PL = P // 2
        WL = int(w[l0:l0 + PL].sum())
        W = int(w[l0:l1].sum())
        nL = (len(idx) * WL) // W
        stack.append((sidx[nL:], l0 + PL, l1))
        stack.append((sidx[:nL], l0, l0 + PL))
    return labels


def graph_bisection(band, n_sub: int, leaf_weights=None) -> np.ndarray:
    """Labels in [0, n_sub) for the actives by recursive bisection of the active 6-neighbour
    graph (the nearest-neighbour graph of Sec. 3.1; reading R-graph).  Breadth-first searches
    stay inside the part and take neighbours in neighbour-table order.  At a tree node:
      a = the node a search from the part's lowest index reaches last, b = the node a search
      from a reaches last; nodes sorted by (d(a, x) - d(b, x), index), nodes a does not reach
      last by index; the first floor(n W_L / W) go left;
      then swap passes (at most 8, until one swaps nothing): each side's nodes with a
      neighbour across and gain = (neighbours across) - (neighbours alongside) >= 0, sorted by
      (-gain, index); the i-th left and i-th right candidates swap when their gains at that
      moment sum, less 2 if they are neighbours, to more than 0."""
    na = band.n_active
    adj = [[int(v) for v in band.nbr[g] if 0 <= v < na] for g in range(na)]
    w = np.ones(n_sub, dtype=np.int64) if leaf_weights is None else np.asarray(leaf_weights, np.int64)
    labels = np.full(na, -1, dtype=np.int64)
    owner = np.zeros(na, dtype=np.int64)          # which part a node is in
    side = np.zeros(na, dtype=np.int64)

    def distances(members, part_id, start):
        """(distance from start or -1 per node, the node reached last)."""
        dist = {int(g): -1 for g in members}
        dist[start] = 0
        q = collections.deque([start])
        last = start
        while q:
            u = q.popleft()
            last = u
            for v in adj[u]:
                if owner[v] == part_id and dist[v] < 0:
                    dist[v] = dist[u] + 1
                    q.append(v)
        return dist, last

    def gain(g, part_id):
        across = sum(1 for v in adj[g] if owner[v] == part_id and side[v] != side[g])
        along = sum(1 for v in adj[g] if owner[v] == part_id and side[v] == side[g])
        return across, across - along

    next_id = 1
    stack = [(np.arange(na, dtype=np.int64), 0, n_sub, 0)]
    while stack:
        members, l0, l1, part_id = stack.pop()
        if l1 - l0 == 1:
            labels[members] = l0
            continue
        if len(members) == 0:
            continue
        _, a = distances(members, part_id, int(members[0]))
        da, b = distances(members, part_id, a)
        db, _ = distances(members, part_id, b)
        far = 1 << 40
        order = sorted((int(g) for g in members),
                       key=lambda g: (da[g] - db[g] if da[g] >= 0 else far, g))
        PL = (l1 - l0) // 2
        WL = int(w[l0:l0 + PL].sum())
        W = int(w[l0:l1].sum())
        nL = (len(members) * WL) // W
        for q, g in enumerate(order):
            side[g] = 0 if q < nL else 1
        for _ in range(8):
            left, right = [], []
            for g in members:
                across, gn = gain(int(g), part_id)
                if across > 0 and gn >= 0:
                    (left if side[g] == 0 else right).append((-gn, int(g)))
            left.sort()
            right.sort()
            swaps = 0
            for (_, u), (_, v) in zip(left, right):
                nb = 1 if v in adj[u] else 0
                if gain(u, part_id)[1] + gain(v, part_id)[1] - 2 * nb > 0:
                    side[u], side[v] = 1, 0
                    swaps += 1
            if swaps == 0:
                break
        lm = members[side[members] == 0]
        rm = members[side[members] == 1]
        owner[lm], owner[rm] = next_id, next_id + 1
        stack.append((rm, l0 + PL, l1, next_id + 1))
        stack.append((lm, l0, l0 + PL, next_id))
        next_id += 2
    return labels


def align_interfaces(band, labels: np.ndarray, passes: int) -> np.ndarray:
    """Labels after `passes` interface-alignment passes (Sec. 3.2)."""
    lab = np.asarray(labels, dtype=np.int64).copy()
    n_a = band.n_active
    near = np.floor(band.cp[:n_a] / band.h + 0.5).astype(np.int64)     # nearest grid point
    target_node = band.lookup(near)
    for _ in range(passes):
        nb = band.nbr                                               # (N_A, 6), ghosts >= n_a
        act = nb < n_a
        nl = np.where(act, lab[np.minimum(nb, n_a - 1)], -1)
        interface = np.any(act & (nl != lab[:, None]), axis=1)
        ok = interface & (target_node >= 0) & (target_node < n_a)
        tgt = np.where(ok, lab[np.clip(target_node, 0, n_a - 1)], lab)
        lab = np.where(ok, tgt, lab)
    return lab


@dataclasses.dataclass
class Subdomain:
    j: int
    own: np.ndarray         # disjoint set  (global active indices, sorted)
    sigma: np.ndarray       # overlapping set Sigma_j (sorted)
    last: np.ndarray        # last overlap layer (sorted)
    ghost: np.ndarray       # Sigma_j^G (global node indices >= N_A, sorted)
    bc_a: np.ndarray        # Sigma_j^{BC} active part (sorted)
    bc_g: np.ndarray        # Robin ghost layer around bc_a (global node indices, sorted)


def bfs_layers(band, labels: np.ndarray, j: int, n_overlap: int) -> np.ndarray:
    """BFS distance (or -1) from the disjoint set j over the active 6-neighbour graph."""
    n_a = band.n_active
    dist = np.full(n_a, -1, dtype=np.int64)
    front = np.flatnonzero(labels == j)
    dist[front] = 0
    for layer in range(1, n_overlap + 1):
        cand = band.nbr[front].ravel()
        cand = np.unique(cand[cand < n_a])
        cand = cand[dist[cand] < 0]
        dist[cand] = layer
        front = cand
    return dist


def stencil_nodes(E, rows: np.ndarray) -> np.ndarray:
    """Union of the interpolation stencils (active columns of E) of the given rows."""
    if len(rows) == 0:
        return np.zeros(0, dtype=np.int64)
    return np.unique(E.tocsr()[rows].indices).astype(np.int64)


def build_subdomain(band, E, labels, j: int, n_overlap: int, robin: bool) -> Subdomain:
    n_a = band.n_active
    dist = bfs_layers(band, labels, j, n_overlap)
    sigma = np.flatnonzero(dist >= 0)
    last = np.flatnonzero(dist == n_overlap)
    in_sigma = dist >= 0
    nb = band.nbr[sigma].ravel()
    ghost = np.unique(nb[nb >= n_a])
    act_nb = np.unique(nb[nb < n_a])
    act_nb = act_nb[~in_sigma[act_nb]]
    sten = stencil_nodes(E, np.concatenate([sigma, ghost]))
    sten = sten[~in_sigma[sten]]
    bc_a = np.union1d(act_nb, sten)
    if robin:
        nb2 = np.unique(band.nbr[bc_a].ravel())
        taken = np.concatenate([sigma, ghost, bc_a])
        bc_g = np.setdiff1d(nb2, taken)
    else:
        bc_g = np.zeros(0, dtype=np.int64)
    return Subdomain(j, np.flatnonzero(labels == j), sigma, last, ghost, bc_a, bc_g)


def cross_point_nodes(band, labels: np.ndarray) -> np.ndarray:
    """Active nodes with active 6-neighbours in >= 2 subdomains other than their own."""
    n_a = band.n_active
    nl = np.where(band.nbr < n_a, labels[np.minimum(band.nbr, n_a - 1)], -1)
    nl = np.where(nl == labels[:, None], -1, nl)
    s = np.sort(nl, axis=1)
    distinct = (s >= 0) & np.concatenate([np.ones((n_a, 1), bool), s[:, 1:] != s[:, :-1]], axis=1)
    return np.flatnonzero(distinct.sum(axis=1) >= 2)


class CrossMarks:
    """Grid nodes within 2 N_O grid steps (Euclidean, inclusive) of any cross-point node."""

    def __init__(self, band, cross: np.ndarray, n_overlap: int):
        self.band = band
        rad = 2 * n_overlap
        self.lo = band.ijk.min(0) - rad
        hi = band.ijk.max(0) + rad
        self.mark = np.zeros(tuple((hi - self.lo + 1).tolist()), dtype=bool)
        if len(cross) == 0:
            return
        r = np.arange(-rad, rad + 1)
        A, B, C = np.meshgrid(r, r, r, indexing="ij")
        ball = np.stack([A.ravel(), B.ravel(), C.ravel()], 1)
        ball = ball[(ball * ball).sum(1) <= rad * rad]
        cij = band.ijk[cross] - self.lo
        for off in ball:                     # dilate the cross points by the integer ball
            q = cij + off
            self.mark[q[:, 0], q[:, 1], q[:, 2]] = True

    def __call__(self, nodes: np.ndarray) -> np.ndarray:
        qn = self.band.ijk[nodes] - self.lo
        return self.mark[qn[:, 0], qn[:, 1], qn[:, 2]]


def effective_boundary_cp(band, sub: Subdomain, nodes: np.ndarray):
    """CP_{S_j}(x) for the given nodes (Eq. locCP, BC line): nearest point of Lambda_j.

    Returns (points (M,3), generator global index (M,))."""
    lam_pts = band.cp[sub.last]
    X = band.coords(nodes)
    best = np.empty(len(nodes), dtype=np.int64)
    for s in range(0, len(nodes), 2048):       # exhaustive argmin in chunks
        Xc = X[s:s + 2048]
        D = Xc[:, None, :] - lam_pts[None, :, :]
        d2 = (D[..., 0] * D[..., 0] + D[..., 1] * D[..., 1]) + D[..., 2] * D[..., 2]
        best[s:s + 2048] = np.argmin(d2, axis=1)   # first minimum = lowest tag
    return lam_pts[best], sub.last[best]


def all_subdomains(band, E, labels, n_sub: int, n_overlap: int, robin: bool):
    return [build_subdomain(band, E, labels, j, n_overlap, robin) for j in range(n_sub)]


__all__ = ["rcb", "Subdomain", "bfs_layers", "build_subdomain", "cross_point_nodes",
           "CrossMarks", "effective_boundary_cp", "all_subdomains", "NBR_OFFSETS"]
