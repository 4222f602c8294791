"""Robin-weight experiment of Sec. 6.3 (Table 2 setting), run on the oracle.

Test infrastructure: decides between the two readings of the Robin local operator's
boundary rows (R1: 7-point rows on every local unknown; R3: (c + 6/h^2) w - (6/h^2) T w on
the boundary unknowns) by the iteration counts the paper reports for the unit sphere split
into two subdomains with overlap N_O = 4, p = 2, h = 1/50, as the solver (Eq. algRAS) and as
the preconditioner, to a 10^6 reduction of the residual 2-norm, over the Robin weight alpha
(alpha = inf is RAS).  There are no cross points with two subdomains.

    python -m oracle.robin_table2 [--h 0.02] [--alphas 0.25,0.5,...] [--align 3] > robin_table2.md

Prints a markdown table of this build's counts beside the paper's.
"""
from __future__ import annotations

import argparse
import math
import time

import numpy as np

from . import krylov, problems, schwarz

# Table 2, h = 1/50 row of the solver and of the preconditioner blocks
PAPER_ALPHAS = [0.25, 0.5, 0.75, 1.0, 1.5, 2.0, 4.0, 8.0, 16.0, math.inf]
PAPER_SOLVER = [19, 14, 11, 11, 15, 20, 33, 49, 67, 83]
PAPER_PRECOND = [11, 9, 9, 8, 8, 9, 11, 13, 15, 17]


def run(h: float, alphas, readings, tol: float = 1e-6, c: float = 1.0, align_passes: int = 0,
        split: str = "coordinate"):
    rows = []
    for a in alphas:
        for rd in (readings if math.isfinite(a) else ["-"]):
            t0 = time.time()
            if math.isfinite(a):
                P = problems.setup("sphere", 1.0, 0.0, h, 2, c, 2, 4, "oras", a, a, reading=rd,
                                   align_passes=align_passes, split=split)
            else:
                P = problems.setup("sphere", 1.0, 0.0, h, 2, c, 2, 4, "ras", align_passes=align_passes,
                                   split=split)
            cp = P.band.cp[:P.band.n_active]
            f = (c + 12.0) * cp[:, 0] * cp[:, 1] * cp[:, 2]
            _, it_s, ok_s = schwarz.stationary_solve(P.A, P.M, f, tol, 2000)
            g = krylov.fgmres(lambda x: P.A @ x, P.M.apply, f, tol, 50, 2000)
            rows.append((a, rd, it_s if ok_s else -1, g.iterations, time.time() - t0))
    return rows


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--h", type=float, default=1.0 / 50)
    ap.add_argument("--alphas", default=",".join(str(a) for a in PAPER_ALPHAS))
    ap.add_argument("--readings", default="R1,R3")
    ap.add_argument("--align", type=int, default=0, help="interface alignment passes (Sec. 3.2)")
    ap.add_argument("--split", default="coordinate", choices=["coordinate", "graph"],
                    help="disjoint split: coordinate or graph bisection")
    args = ap.parse_args()
    alphas = [float(x) for x in args.alphas.split(",")]
    rows = run(args.h, alphas, args.readings.split(","), align_passes=args.align, split=args.split)
    paper = dict(zip(PAPER_ALPHAS, zip(PAPER_SOLVER, PAPER_PRECOND)))
    print(f"unit sphere, p = 2, h = {args.h:g}, 2 subdomains ({args.split} bisection), N_O = 4, "
          f"{args.align} alignment passes, 1e6 reduction\n")
    print("| alpha | reading | solver (paper) | solver (oracle) | preconditioner (paper) | "
          "preconditioner (oracle, right-preconditioned FGMRES) | set-up + solves s |")
    print("|---|---|---|---|---|---|---|")
    for a, rd, s_it, g_it, sec in rows:
        ps, pp = paper.get(a, ("", ""))
        name = "inf (RAS)" if not math.isfinite(a) else f"{a:g}"
        print(f"| {name} | {rd} | {ps} | {s_it} | {pp} | {g_it} | {sec:.0f} |", flush=True)


if __name__ == "__main__":
    main()
