"""Closest-point functions CP_S and surface normals (Sec. 2.1, definition of CP_S).

CP_S(x) = argmin_{y in S} ||x - y||_2.  For the sphere and the torus it has a closed form.
All arithmetic is FP64 in a fixed operation order (norms as sqrt((x*x + y*y) + z*z)).
"""
from __future__ import annotations

import numpy as np


def norm3(V: np.ndarray) -> np.ndarray:
    """Euclidean norm of rows of an (N, 3) array, summed x, then y, then z."""
    return np.sqrt((V[:, 0] * V[:, 0] + V[:, 1] * V[:, 1]) + V[:, 2] * V[:, 2])


class Sphere:
    """Sphere of radius R centred at the origin: CP(x) = R x/|x|."""

    kind = "sphere"

    def __init__(self, R: float = 1.0):
        self.R = float(R)

    def bbox(self):
        R = self.R
        return np.array([-R, -R, -R]), np.array([R, R, R])

    def cp(self, X: np.ndarray) -> np.ndarray:
        X = np.asarray(X, dtype=np.float64)
        r = norm3(X)
        with np.errstate(divide="ignore", invalid="ignore"):
            Y = (X / r[:, None]) * self.R
        Y[r == 0.0] = np.nan          # CP undefined at the centre: never in the band
        return Y

    def normal(self, Y: np.ndarray) -> np.ndarray:
        """Unit outward normal at surface points Y."""
        return Y / norm3(Y)[:, None]

    def radial_bounds(self):
        """The set of x with ||x - CP(x)|| <= d is the shell | |x| - R | <= d."""
        return self.R


class Torus:
    """Torus about the z axis with major radius R and minor radius r.

    The ring circle is C(x) = R (x, y, 0)/rho with rho = sqrt(x^2 + y^2); then
    CP(x) = C + r (x - C)/|x - C|.
    """

    kind = "torus"

    def __init__(self, R: float = 1.0, r: float = 0.4):
        self.R = float(R)
        self.r = float(r)

    def bbox(self):
        a = self.R + self.r
        return np.array([-a, -a, -self.r]), np.array([a, a, self.r])

    def _ring(self, X: np.ndarray) -> np.ndarray:
        rho = np.sqrt(X[:, 0] * X[:, 0] + X[:, 1] * X[:, 1])
        C = np.zeros_like(X)
        with np.errstate(divide="ignore", invalid="ignore"):
            C[:, 0] = (X[:, 0] / rho) * self.R
            C[:, 1] = (X[:, 1] / rho) * self.R
        C[rho == 0.0] = np.nan        # CP undefined on the axis: never in the band
        return C

    def cp(self, X: np.ndarray) -> np.ndarray:
        X = np.asarray(X, dtype=np.float64)
        C = self._ring(X)
        V = X - C
        s = norm3(V)
        with np.errstate(divide="ignore", invalid="ignore"):
            Y = C + (V / s[:, None]) * self.r
        Y[s == 0.0] = np.nan          # CP undefined on the ring circle itself
        return Y

    def normal(self, Y: np.ndarray) -> np.ndarray:
        C = self._ring(Y)
        V = Y - C
        return V / norm3(V)[:, None]


def make_surface(kind: str, R: float, r: float = 0.0):
    if kind == "sphere":
        return Sphere(R)
    if kind == "torus":
        return Torus(R, r)
    raise ValueError(kind)
