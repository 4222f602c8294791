"""Right-preconditioned flexible GMRES(m) (Saad's FGMRES) with CGS2 (Sec. 2.2, Sec. 6.6).

The paper embeds (O)RAS in GMRES without naming side, orthogonalisation or restart; this
oracle fixes them (readings): right preconditioning with the flexible basis Z, classical
Gram-Schmidt applied twice, Givens rotations, restart length m, x0 = 0.

One cycle from x with r = f - A x, beta = ||r||:
  v_0 = r / beta,  g = beta e_0
  for k = 0, 1, ...:
      z_k = M^{-1} v_k,  w = A z_k
      h  = V_k^T w ;  w = w - V_k h          (first Gram-Schmidt pass)
      h2 = V_k^T w ;  w = w - V_k h2 ;  h += h2   (second pass)
      H[k+1, k] = ||w|| ;  v_{k+1} = w / ||w||
      rotate column k of H by the previous Givens rotations, build rotation k from
      (H[k,k], H[k+1,k]) with rho = sqrt(a^2 + b^2), c = a/rho, s = b/rho, and update
      g[k+1] = -s g[k], g[k] = c g[k]
      stop the cycle when |g[k+1]| <= tol ||f||, at m steps, or at breakdown (||w|| = 0)
  y = H[:k+1, :k+1]^{-1} g[:k+1] (back substitution),  x = x + Z_k y
Then the true residual ||f - A x|| decides convergence (<= tol ||f||); otherwise restart.

Breakdown (a reading; the paper never meets it): ||w|| = 0 means A z_k lies in the span of
the basis.  If the rotated diagonal rho is nonzero the least-squares problem is solved
exactly (a "happy" breakdown) and the cycle ends as usual.  If rho = 0 the Hessenberg matrix
is singular: column k is left out (the update uses the first k columns) and the solve stops.
In both cases a true residual still above the tolerance ends the solve with breakdown set,
since restarting from the same residual would build the same basis again.
"""
from __future__ import annotations

import dataclasses

import numpy as np


@dataclasses.dataclass
class GmresResult:
    x: np.ndarray
    iterations: int
    relres: float
    converged: bool
    history: list          # |g_{k+1}| / ||f|| after every inner step
    breakdown: bool = False


def fgmres(A_apply, M_apply, f: np.ndarray, tol: float, restart: int = 50,
           max_it: int = 1000, x0: np.ndarray | None = None, stop_after: int | None = None):
    """stop_after: end after exactly this many inner iterations (for iterate comparisons)."""
    n = len(f)
    nf = float(np.sqrt(f @ f))
    x = np.zeros(n) if x0 is None else x0.copy()
    hist = []
    if nf == 0.0:
        return GmresResult(np.zeros(n), 0, 0.0, True, hist)
    total = 0
    r = f - A_apply(x)
    beta = float(np.sqrt(r @ r))
    while True:
        m = restart
        V = np.zeros((m + 1, n))
        Z = np.zeros((m, n))
        H = np.zeros((m + 1, m))
        cs = np.zeros(m)
        sn = np.zeros(m)
        g = np.zeros(m + 1)
        g[0] = beta
        V[0] = r / beta
        k_done = 0
        broke = False
        for k in range(m):
            Z[k] = M_apply(V[k])
            w = A_apply(Z[k])
            h = V[:k + 1] @ w
            w = w - V[:k + 1].T @ h
            h2 = V[:k + 1] @ w
            w = w - V[:k + 1].T @ h2
            h = h + h2
            hn = float(np.sqrt(w @ w))
            H[:k + 1, k] = h
            H[k + 1, k] = hn
            if hn > 0.0:
                V[k + 1] = w / hn
            for i in range(k):
                t = cs[i] * H[i, k] + sn[i] * H[i + 1, k]
                H[i + 1, k] = -sn[i] * H[i, k] + cs[i] * H[i + 1, k]
                H[i, k] = t
            a, b = H[k, k], H[k + 1, k]
            rho = np.sqrt(a * a + b * b)
            total += 1
            if rho == 0.0:                 # singular Hessenberg: drop column k
                broke = True
                k_done = k
                hist.append(abs(g[k]) / nf)
                break
            cs[k], sn[k] = a / rho, b / rho
            H[k, k] = rho
            H[k + 1, k] = 0.0
            g[k + 1] = -sn[k] * g[k]
            g[k] = cs[k] * g[k]
            k_done = k + 1
            hist.append(abs(g[k + 1]) / nf)
            if hn == 0.0:
                broke = True
                break
            if abs(g[k + 1]) <= tol * nf or total >= max_it:
                break
            if stop_after is not None and total >= stop_after:
                break
        y = np.zeros(k_done)
        for i in range(k_done - 1, -1, -1):
            y[i] = (g[i] - H[i, i + 1:k_done] @ y[i + 1:]) / H[i, i]
        x = x + Z[:k_done].T @ y
        r = f - A_apply(x)
        beta = float(np.sqrt(r @ r))
        rel = beta / nf
        if stop_after is not None and total >= stop_after:
            return GmresResult(x, total, rel, rel <= tol, hist)
        if rel <= tol:
            return GmresResult(x, total, rel, True, hist)
        if total >= max_it or beta == 0.0:
            return GmresResult(x, total, rel, False, hist)
        if broke:
            return GmresResult(x, total, rel, False, hist, True)
