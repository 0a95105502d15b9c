"""Comparison of converged equilibria and their properties (test infrastructure only).

* Translations (§5: plane Couette flow is equivariant under continuous shifts in x and z,
  so every equilibrium comes with a two-parameter family of shifted copies, all with
  J = 0).  ``shift`` moves a spectral field by (lx, lz): a(x - lx, y, z - lz).
  ``align`` finds the shift of b that is closest to a in the norm of J, so that two
  converged equilibria of the same family can be compared element by element.
* Table 2's properties: the volume-normalised L2 norm ||u|| and the total dissipation
  D/D_lam = (1/V) int |grad(u_b + u)|^2 dV / (1/V) int |grad u_b|^2 dV, V = 2 Lx Lz.
  For u_b = (y, 0, 0), |grad u_b|^2 = 1, and the cross term 2 int d_y u_x vanishes
  because u = 0 at the walls, so D/D_lam = 1 + ||grad u||^2 in the same normalisation.
"""
import math

import numpy as np


def shift(o, a, lx, lz):
    """Spectral field of a(x - lx, y, z - lz) for an oracle ``o``'s grid."""
    ph = np.exp(-1j * (o.kx[:, None] * lx + o.kz[None, :] * lz))
    return a * ph[None, :, :, None]


def _mode_correlation(o, a, b):
    """c[m, p] with  (1/(2 Lx Lz)) int a . shift(b, lx, lz) = Re sum c[m, p] e^{-i(kx lx + kz lz)}.

    The mean over x, z of the product of two real fields is the sum over all (m, p) of
    conj(a_mp) b_mp; the stored half p >= 0 counts the p > 0 modes twice.  In y the
    integral uses the Clenshaw-Curtis weights at the Gauss-Lobatto points (values = C @ coeffs)."""
    av = a @ o.C.T
    bv = b @ o.C.T
    c = 0.5 * (np.conj(av) * bv * o.w_cc).sum(axis=(0, -1))
    c[:, 1:] *= 2.0
    return c


def align(o, a, b, grid=64, newton_steps=50):
    """Shift (lx, lz) that minimises ||a - shift(b, lx, lz)||, the shifted b, and the
    relative distance ||a - shift(b)|| / ||a||.  The correlation is sampled on a
    grid x grid lattice of shifts over one period; Newton's method on its analytic
    gradient and Hessian then refines the best lattice point (function values alone
    cannot place a maximum closer than about sqrt(machine epsilon))."""
    c = _mode_correlation(o, a, b)
    KX = np.broadcast_to(o.kx[:, None], c.shape)
    KZ = np.broadcast_to(o.kz[None, :], c.shape)

    def terms(s):
        return c * np.exp(-1j * (KX * s[0] + KZ * s[1]))
    best, arg = -math.inf, np.zeros(2)
    for i in range(grid):
        for j in range(grid):
            s = np.array([o.Lx * i / grid, o.Lz * j / grid])
            v = float(np.real(terms(s).sum()))
            if v > best:
                best, arg = v, s
    s = arg.copy()
    for _ in range(newton_steps):
        t = terms(s)
        g = np.array([np.real((-1j * KX * t).sum()), np.real((-1j * KZ * t).sum())])
        H = -np.array([[np.real((KX * KX * t).sum()), np.real((KX * KZ * t).sum())],
                       [np.real((KX * KZ * t).sum()), np.real((KZ * KZ * t).sum())]])
        if not np.all(np.linalg.eigvalsh(H) < 0):
            break
        step = -np.linalg.solve(H, g)
        s = s + step
        if np.max(np.abs(step)) < 1e-15 * max(o.Lx, o.Lz):
            break
    lx, lz = float(s[0]) % o.Lx, float(s[1]) % o.Lz
    bs = shift(o, b, lx, lz)
    na = o.norm(a)
    return lx, lz, bs, o.norm(a - bs) / (na if na > 0 else 1.0)


def dissipation(o, a):
    """D / D_lam of u_b + a with u_b = (y, 0, 0) (Table 2's second property)."""
    _, grad = o.fields(a)
    g = grad.reshape((9,) + grad.shape[2:])
    s = (g ** 2).sum(axis=0).mean(axis=(-2, -1))
    return 1.0 + 0.5 * float((o.w_cc * s).sum())
