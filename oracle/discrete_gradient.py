"""Exact gradient of the discrete cost, for checking the paper's descent direction
(test infrastructure only).

The method minimises J = ||r1|| (Fig. 1 caption) by the adjoint dynamics of §3, which it
discretises in §4: the direction f of Eq. (f_approximation) is a finite-difference,
Stokes-preconditioned approximation of the adjoint, not the exact gradient of the
discrete cost J_h(u) = 1/2 ||r1(u)||^2 that the discretised residual map defines.  This
module computes that exact gradient g_h = (d r1/du)^T W r1 by transposing the discrete
chain of §4 steps 1-2 (synthesis, products, analysis, Stokes solve, quotient, norm):
it restates the oracle's residual with PyTorch CPU operations in FP64 (the same
definitions: the same collocation matrices, the 2/3-truncated FFTs, the products M of
Eq. (u_trick), the dense tau systems of every mode, Clenshaw-Curtis weights) and lets
reverse-mode differentiation apply the transposed stages.

Inner product of the gradient: for complex coefficient arrays g, v of the uhat layout,
<g, v> = sum Re(conj(g) v), i.e. g = dJ_h/dRe(u) + i dJ_h/dIm(u), so that <g_h, v> is
the derivative of J_h along v.
"""
import numpy as np
import torch


class DiscreteCost:
    """J_h and its exact gradient on the grid of a PCFOracle ``o``."""

    def __init__(self, o):
        self.o = o
        t = lambda a: torch.tensor(a, dtype=torch.float64)  # noqa: E731
        self.C = t(o.C)
        self.Cinv = t(o.Cinv)
        self.w = t(o.w_cc)
        self.KX = torch.tensor(o.kx, dtype=torch.complex128)[:, None, None]
        self.KZ = torch.tensor(o.kz, dtype=torch.complex128)[None, :, None]
        self.D = t(o.Dmat)
        self.xi = torch.tensor(o.x_index)
        self.U = t(o.U_phys)
        self.dU = t(o.dU_phys)
        self.V = float(o.V_base)
        self._sys = {}

    # ---------------------------------------------------------------- the oracle's stages, in torch
    def to_phys(self, a):
        vals = torch.movedim(a @ self.C.T.to(a.dtype), -1, -3)
        o = self.o
        full = torch.zeros(vals.shape[:-2] + (o.nx, o.nz // 2 + 1), dtype=torch.complex128)
        full[..., self.xi, : o.Mz] = vals
        return torch.fft.irfft2(full, s=(o.nx, o.nz), norm="forward")

    def to_spec(self, f):
        o = self.o
        F = torch.fft.rfft2(f, norm="forward")[..., self.xi, : o.Mz]
        return torch.movedim(F, -3, -1) @ self.Cinv.T.to(torch.complex128)

    def fields(self, a):
        val = self.to_phys(a)
        D = self.D.T.to(torch.complex128)
        grads = []
        for i in range(3):
            grads.append(torch.stack([self.to_phys(1j * self.KX * a[i]), self.to_phys(a[i] @ D),
                                      self.to_phys(1j * self.KZ * a[i])]))
        return val, torch.stack(grads)

    def M_hat(self, u, g):
        out = []
        for i in range(3):
            conv = u[0] * g[i, 0] + u[1] * g[i, 1] + u[2] * g[i, 2]
            m = -self.U * g[i, 0] - self.V * g[i, 1] - conv
            if i == 0:
                m = m - self.dU * u[1]
            out.append(m)
        return self.to_spec(torch.stack(out))

    def _systems(self, sigma):
        key = float(sigma)
        if key not in self._sys:
            tab = {}
            for ij, (A, scale) in self.o.stokes_systems(sigma).items():
                if scale is None:
                    tab[ij] = (torch.tensor(A, dtype=torch.complex128), None)
                else:
                    tab[ij] = (torch.tensor(A * scale[:, None], dtype=torch.complex128),
                               torch.tensor(scale, dtype=torch.complex128))
            self._sys[key] = tab
        return self._sys[key]

    def stokes_step(self, rhs, step):
        """(1/step - nu Lap) w + grad p = rhs, div w = 0, w(+-1) = 0: the oracle's dense tau
        systems, solved per mode."""
        o = self.o
        sigma = 1.0 / (o.nu * step)
        F = rhs / o.nu
        N, n1 = o.N, o.N + 1
        out = torch.zeros_like(F)
        for (i, j), (A, scale) in self._systems(sigma).items():
            if scale is None:
                for c in (0, 2):
                    b = torch.zeros(n1, dtype=torch.complex128)
                    b[: N - 1] = F[c, i, j, : N - 1]
                    out[c, i, j] = torch.linalg.solve(A, b)
                continue
            b = torch.zeros(4 * n1, dtype=torch.complex128)
            for c in range(3):
                b[c * (N - 1):(c + 1) * (N - 1)] = F[c, i, j, : N - 1]
            x = torch.linalg.solve(A, b * scale)
            for c in range(3):
                out[c, i, j] = x[c * n1:(c + 1) * n1]
        return out

    def residual(self, u):
        o = self.o
        val, g = self.fields(u)
        u_dt = self.stokes_step(u / o.dt + self.M_hat(val, g), o.dt)
        return (u_dt - u) / o.dt

    def half_J2(self, u):
        """J_h = 1/2 ||r1||^2 with the oracle's norm (a torch scalar)."""
        r = self.residual(u)
        s = (self.to_phys(r) ** 2).sum(dim=0).mean(dim=(-2, -1))
        return 0.25 * (self.w * s).sum()

    # ---------------------------------------------------------------- numpy interface
    def value(self, u):
        with torch.no_grad():
            return float(self.half_J2(torch.tensor(u, dtype=torch.complex128)))

    def gradient(self, u):
        """g_h = dJ_h/dRe(u) + i dJ_h/dIm(u) (numpy complex, the uhat layout)."""
        re = torch.tensor(np.real(u), dtype=torch.float64, requires_grad=True)
        im = torch.tensor(np.imag(u), dtype=torch.float64, requires_grad=True)
        J = self.half_J2(torch.complex(re, im))
        gre, gim = torch.autograd.grad(J, (re, im))
        return gre.numpy() + 1j * gim.numpy()


def inner(g, v):
    """<g, v> = sum Re(conj(g) v): the derivative of J_h along v when g is its gradient."""
    return float(np.sum(np.real(np.conj(g) * v)))


def central_difference(cost, u, v, eps):
    """(J_h(u + eps v) - J_h(u - eps v)) / (2 eps)."""
    return (cost.value(u + eps * v) - cost.value(u - eps * v)) / (2.0 * eps)

