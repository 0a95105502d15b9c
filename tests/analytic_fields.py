"""Exactly integrable trigonometric-polynomial fields for the continuous-level pins.

Fields are evaluated (with their first and second derivatives) by numpy's Chebyshev
routines on an over-resolved quadrature grid: uniform in x and z (exact for the
trigonometric degrees that occur) and Gauss-Legendre in y (exact for the polynomial
degrees that occur).  Nothing here comes from the oracle.
"""
import math

import numpy as np
from numpy.polynomial import chebyshev as C

WALL = {0: np.array([1.0]), 1: np.array([0.5, 0.0, -0.5])}   # 1, (1 - y^2)
WALL[2] = C.chebmul(WALL[1], WALL[1])                           # (1 - y^2)^2


class Grid:
    def __init__(self, Lx, Lz, nf=12, ng=24):
        self.Lx, self.Lz = Lx, Lz
        self.x = np.arange(nf) * Lx / nf
        self.z = np.arange(nf) * Lz / nf
        yg, wg = np.polynomial.legendre.leggauss(ng)
        self.y, self.wy = yg, wg
        self.Y = yg[:, None, None]
        self.nf = nf

    def integrate(self, f):
        """int over the box of f given on (ng, nf, nf)."""
        return float((self.wy[:, None, None] * f).sum()) * self.Lx * self.Lz / self.nf ** 2


class Scalar:
    """f = sum_{m,p} Re-combination of c_{m,p}(y) exp(i(kx x + kz z)), real-valued."""

    def __init__(self, coef, wall, K, Lx, Lz):
        self.coef = coef          # complex (2K+1, K+1, n0) Chebyshev coefficients before the wall factor
        self.wall = wall
        self.K, self.Lx, self.Lz = K, Lx, Lz

    @staticmethod
    def random(rng, K, n0, wall, Lx, Lz, scale=1.0):
        c = scale * (rng.standard_normal((2 * K + 1, K + 1, n0)) + 1j * rng.standard_normal((2 * K + 1, K + 1, n0)))
        c[0, 0] = c[0, 0].real
        for i in range(1, K + 1):       # p = 0 plane conjugate-symmetric in m
            c[2 * K + 1 - i, 0] = np.conj(c[i, 0])
        return Scalar(c, wall, K, Lx, Lz)

    def __add__(self, o):
        assert self.wall == o.wall
        return Scalar(self.coef + o.coef, self.wall, self.K, self.Lx, self.Lz)

    def scaled(self, a):
        return Scalar(a * self.coef, self.wall, self.K, self.Lx, self.Lz)

    def _modes(self):
        K = self.K
        ms = list(range(K + 1)) + list(range(-K, 0))
        for i, m in enumerate(ms):
            for p in range(K + 1):
                yield i, p, 2 * math.pi * m / self.Lx, 2 * math.pi * p / self.Lz, (1.0 if p == 0 else 2.0)

    def eval(self, g):
        """Returns dict with value, first derivatives (x, y, z) and Laplacian on grid g."""
        X = g.x[None, :, None]
        Z = g.z[None, None, :]
        shape = (len(g.y), len(g.x), len(g.z))
        out = {k: np.zeros(shape) for k in ("f", "fx", "fy", "fz", "lap")}
        for i, p, kx, kz, w in self._modes():
            prof = C.chebmul(self.coef[i, p], WALL[self.wall])
            d1 = C.chebder(prof)
            d2 = C.chebder(prof, 2)
            P0 = C.chebval(g.y, prof)[:, None, None]
            P1 = C.chebval(g.y, d1)[:, None, None]
            P2 = C.chebval(g.y, d2)[:, None, None]
            E = np.exp(1j * (kx * X + kz * Z))
            out["f"] += w * np.real(P0 * E)
            out["fx"] += w * np.real(1j * kx * P0 * E)
            out["fy"] += w * np.real(P1 * E)
            out["fz"] += w * np.real(1j * kz * P0 * E)
            out["lap"] += w * np.real((P2 - (kx * kx + kz * kz) * P0) * E)
        return out


def vector_eval(comps, g):
    """(values (3,...), gradient (3,3,...) with [i, j] = d_j f_i, Laplacian (3,...))."""
    ev = [c.eval(g) for c in comps]
    val = np.stack([e["f"] for e in ev])
    grad = np.stack([np.stack([e["fx"], e["fy"], e["fz"]]) for e in ev])
    lap = np.stack([e["lap"] for e in ev])
    return val, grad, lap
