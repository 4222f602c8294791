"""Oracle local solves of many subdomains in spawned worker processes (test helper).

Each worker builds the oracle's band, extension matrix, partition and cross-point marks of one
workload once (the oracle is deterministic, so every worker holds the same objects), then
assembles the local operator A_j of each subdomain it is given (Eq. localOP / simpleRAS),
factors it with SuperLU and returns z_j on the disjoint set for the right-hand side [R_j r; 0].
"""
from __future__ import annotations

import numpy as np
import scipy.sparse.linalg as spla

_S = {}


def init(name: str, r: np.ndarray):
    from oracle import band as band_mod
    from oracle import geometry, interp, partition
    from workloads import WORKLOADS, leaf_weights
    wl = WORKLOADS[name]
    B = band_mod.build_band(geometry.make_surface(wl.surface, wl.R, wl.r), wl.h, wl.p)
    E = interp.extension_matrix(B)
    labels = partition.rcb(B.cp[: B.n_active], wl.n_sub, leaf_weights(wl.n_sub, wl.weight_seed))
    marks = partition.CrossMarks(B, partition.cross_point_nodes(B, labels), wl.n_overlap)
    A = None
    if wl.method == "ras":
        from oracle import operator
        A = operator.cpm_matrix(B, E, wl.c)
    _S.update(wl=wl, B=B, E=E, labels=labels, marks=marks, A=A, r=r)


def local_solutions(js):
    from oracle import local, partition
    wl, B, E = _S["wl"], _S["B"], _S["E"]
    out = []
    for j in js:
        sub = partition.build_subdomain(B, E, _S["labels"], j, wl.n_overlap, wl.method == "oras")
        if wl.method == "ras":
            lp = local.ras_local(_S["A"], sub)
        else:
            lp = local.oras_local(B, sub, wl.c, wl.alpha, wl.alpha_x, _S["marks"], "R1")
        e = spla.splu(lp.A.tocsc()).solve(lp.rhs(_S["r"]))
        out.append((j, lp.n, lp.own_global, e[lp.own_local]))
    return out


def all_local_solutions(name: str, r: np.ndarray, n_sub: int, workers: int):
    """[(j, n_j, disjoint global indices, oracle z_j there)] for every subdomain j."""
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    chunks = [list(range(k, n_sub, workers * 4)) for k in range(workers * 4)]
    with ctx.Pool(workers, initializer=init, initargs=(name, r)) as pool:
        res = pool.map(local_solutions, [c for c in chunks if c])
    return sorted((x for part in res for x in part), key=lambda t: t[0])
