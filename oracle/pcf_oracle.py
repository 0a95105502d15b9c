"""Plain FP64 CPU oracle of one adjoint-descent step for plane Couette flow.

Test infrastructure only (see ``oracle/__init__.py``); slow and direct on purpose.

What it computes (Ashtari & Schneider, arXiv 2306.00165):

* Discretisation, §4 Eq. (Foureir_Chebyshev_Fourier): u_j(x,y,z) = sum over retained
  (m, p, n) of uhat_{m,p,n,j} T_n(y) exp(2 pi i (m x/Lx + p z/Lz)).  Retained modes
  |m| <= Kx = Nx//3 - 1, 0 <= p <= Kz = Nz//3 - 1 (2/3 rule in x and z, none in y).
  Collocation: y_j = cos(pi j/N), j = 0..N (N = Ny - 1); x, z uniform.
* Nonlinear terms pseudo-spectrally in the convective forms written in the paper:
  M(u) = -(u_b.grad)u - (u.grad)u_b - (u.grad)u with u_b = (y, 0, 0) for plane Couette
  flow (other base flows: base_profile) (§4 Eq. (u_trick), §5), and N(q) = (grad q)(u_b + u) - (grad(u_b + u))^T q  (§4, below Eq. (g_trick)),
  read as component i: U_j d_j q_i - q_j d_i U_j with U = u_b + u.
* Stokes step (the influence-matrix algorithm's discrete target, §4): per mode
  (m, p) != (0, 0), unknowns u, v, w, P in span{T_0..T_N} with
      (sigma + k^2 - D^2) u_c + (grad_k P)_c = F_c   on Chebyshev rows 0..N-2 (c = x, y, z)
      u = v = w = 0 at y = +-1                       (6 rows)
      i kx u + D v + i kz w = 0                       on all rows 0..N
  solved by a dense LU of this (4N+4)^2 system; the mean mode has v = 0 and Dirichlet
  Helmholtz problems for u and w (no mean pressure gradient in plane Couette flow).
* One descent step, §4 steps 1-5:
  1. u^dt  = Stokes step of the NSE (IMEX Euler: implicit viscous term and pressure,
     explicit M), sigma = 1/(nu dt)                      -- Eq. (u_trick)
  2. r1    = (u^dt - u)/dt                                -- Eq. (r1_approximation)
  3. r1^+  = Stokes step of the dummy dynamics with N(r1) in place of M, taken as the
     well-posed (diffusive) direction in tau-hat, sigma = 1/(nu dtau_hat)
  4. f     = -(r1^+ - r1)/dtau_hat                        -- Eq. (f_approximation), sign
     reading: the limit dtau_hat -> 0 gives Eq. (adjoint_evolution_divergence_free)
  5. u    <- u + dtau f                                   -- Eq. (forward_Euler_update)
* Cost J = ||r1|| with the volume-normalised L2 norm (1/(2 Lx Lz)) int |r1|^2,
  Clenshaw-Curtis weights in y and the uniform mean in x, z (§2, Fig. 1: J = ||r(u)||).
* Symmetries of §5.1: s1 [u,v,w](x,y,z) = [-u,-v,w](-x+Lx/2, -y, z+Lz/2) and
  s2 [u,v,w](x,y,z) = [u,v,-w](x+Lx/2, y, -z), applied literally on the collocation grid
  (each is an exact permutation of the grid points there).  The symmetric subspace of a
  set of them is the image of the group average (§3.4: the descent preserves it).
* Direct numerical simulation for the guesses of §5.2: the Stokes step of step 1 used as
  a time stepper, u <- u^dt = u + dt r1, with the local extrema in time of ||u|| taken as
  guesses (discrete extrema: (h_s - h_{s-1}) (h_{s+1} - h_s) < 0).
"""
import math

import numpy as np
import scipy.linalg as sla

TWO_PI = 2.0 * math.pi


def cheb_deriv(a):
    """Chebyshev coefficients of d/dy along the last axis (exact for polynomials).

    Backward recurrence c_{n-1} b_{n-1} = b_{n+1} + 2 n a_n with b_N = b_{N+1} = 0.
    """
    N = a.shape[-1] - 1
    b = np.zeros(a.shape, dtype=np.result_type(a, np.float64))
    if N >= 1:
        b[..., N - 1] = 2.0 * N * a[..., N]
    for n in range(N - 2, -1, -1):
        b[..., n] = b[..., n + 2] + 2.0 * (n + 1) * a[..., n + 1]
    b[..., 0] *= 0.5
    return b


def clenshaw_curtis_weights(N):
    """Weights w_j with sum_j w_j f(cos(pi j/N)) = int_{-1}^{1} f dy for deg f <= N."""
    theta = math.pi * np.arange(N + 1) / N
    w = np.zeros(N + 1)
    for j in range(N + 1):
        s = 0.0
        for k in range(1, N // 2 + 1):
            bk = 1.0 if (2 * k == N) else 2.0
            s += bk / (4.0 * k * k - 1.0) * math.cos(2.0 * k * theta[j])
        cj = 1.0 if j in (0, N) else 2.0
        w[j] = cj / N * (1.0 - s)
    return w


def base_profile(kind, y, nu=None, delta=None):
    """Laminar base flow u_b = (U(y), V, 0): returns U(y), U'(y) and the constant wall-normal
    velocity V (§3.1: the method is derived for a general u_b; §7 names plane Poiseuille and
    the asymptotic suction boundary layer as flows where only u_b changes).
    couette: U = y, V = 0 (walls moving at +-1); poiseuille: U = 1 - y^2, V = 0 (driven by a
    fixed pressure gradient that the base flow absorbs); asbl: the asymptotic suction
    boundary layer over the wall y = -1, U = 1 - exp(-(1 + y)/delta) with uniform suction
    V = -nu/delta (delta: suction length in units of the half-height), which solves
    V U' = nu U'' with no pressure gradient; the wall y = +1 moves at U(1) with the same
    uniform wall-normal velocity."""
    if kind == "couette":
        return y, np.ones_like(y), 0.0
    if kind == "poiseuille":
        return 1.0 - y * y, -2.0 * y, 0.0
    if kind == "asbl":
        if nu is None or delta is None or not delta > 0:
            raise ValueError("asbl needs nu and a suction length delta > 0")
        e = np.exp(-(1.0 + y) / delta)
        return 1.0 - e, e / delta, -nu / delta
    raise ValueError(kind)


def nonlinear_M(u, gu, U, dU=1.0, V=0.0):
    """M(u) = -(u_b.grad) u - (u.grad) u_b - (u.grad) u = -U d_x u - V d_y u - U' v e_x
    - (u.grad) u, pointwise, for u_b = (U(y), V, 0) with V constant.

    u: (3, ...) velocity values; gu: (3, 3, ...) with gu[i, j] = d_j u_i; U, dU broadcastable.
    """
    out = np.empty_like(u)
    for i in range(3):
        conv = u[0] * gu[i, 0] + u[1] * gu[i, 1] + u[2] * gu[i, 2]
        out[i] = -U * gu[i, 0] - V * gu[i, 1] - conv
    out[0] = out[0] - dU * u[1]
    return out


def adjoint_N(q, gq, u, gu, U, dU=1.0, V=0.0):
    """N(q) = (W.grad) q - (grad W)^T q with W = u_b + u = (U(y), V, 0) + u, pointwise.

    Component i: W_j d_j q_i - q_j d_i W_j, where d_i W_j = d_i u_j + delta_{j x} delta_{i y} U'
    (V is constant and adds no gradient).
    """
    U0 = u[0] + U
    V0 = u[1] + V
    out = np.empty_like(q)
    for i in range(3):
        adv = U0 * gq[i, 0] + V0 * gq[i, 1] + u[2] * gq[i, 2]
        tr = q[0] * gu[0, i] + q[1] * gu[1, i] + q[2] * gu[2, i]
        out[i] = adv - tr
    out[1] = out[1] - dU * q[0]
    return out


class PCFOracle:
    """Oracle for one grid; all state arrays are complex128 [3][Mx][Mz][Ny]."""

    def __init__(self, nx, ny, nz, Lx=TWO_PI / 1.14, Lz=TWO_PI / 2.5, Re=400.0,
                 dt=0.25, dtau_hat=0.25, base_flow="couette", suction_length=None):
        self.nx, self.ny, self.nz = nx, ny, nz
        self.Lx, self.Lz, self.Re = float(Lx), float(Lz), float(Re)
        self.nu = 1.0 / self.Re
        self.dt, self.dtau_hat = float(dt), float(dtau_hat)
        self.N = ny - 1
        self.Kx, self.Kz = nx // 3 - 1, nz // 3 - 1
        self.Mx, self.Mz = 2 * self.Kx + 1, self.Kz + 1
        self.m = np.array(list(range(self.Kx + 1)) + list(range(-self.Kx, 0)))
        self.p = np.arange(self.Mz)
        self.kx = TWO_PI * self.m / self.Lx
        self.kz = TWO_PI * self.p / self.Lz
        self.KX = self.kx[:, None, None]
        self.KZ = self.kz[None, :, None]
        self.x_index = self.m % nx            # storage index -> FFT bin in x
        n = np.arange(self.N + 1)
        self.y = np.cos(math.pi * n / self.N)
        # values at the Gauss-Lobatto points = C @ coefficients, C_jn = T_n(y_j)
        self.C = np.cos(math.pi * np.outer(n, n) / self.N)
        self.Cinv = np.linalg.inv(self.C)
        self.w_cc = clenshaw_curtis_weights(self.N)
        self.Dmat = np.stack([cheb_deriv(e) for e in np.eye(self.N + 1)], axis=1)
        self._lu = {}
        self.y_phys = self.y[:, None, None]   # broadcast over (Ny, Nx, Nz)
        self.base_flow = base_flow
        self.suction_length = suction_length
        Ub, dUb, self.V_base = base_profile(base_flow, self.y, self.nu, suction_length)
        self.U_phys, self.dU_phys = Ub[:, None, None], dUb[:, None, None]

    # ---------------------------------------------------------------- transforms
    def to_phys(self, a):
        """Coefficients (..., Mx, Mz, Ny) -> real values (..., Ny, Nx, Nz)."""
        vals = np.moveaxis(a @ self.C.T, -1, -3)
        full = np.zeros(vals.shape[:-2] + (self.nx, self.nz // 2 + 1), np.complex128)
        full[..., self.x_index, : self.Mz] = vals
        return np.fft.irfft2(full, s=(self.nx, self.nz), norm="forward")

    def to_spec(self, f):
        """Real values (..., Ny, Nx, Nz) -> retained coefficients (..., Mx, Mz, Ny)."""
        F = np.fft.rfft2(f, norm="forward")[..., self.x_index, : self.Mz]
        return np.moveaxis(F, -3, -1) @ self.Cinv.T

    def dx(self, a):
        return 1j * self.KX * a

    def dz(self, a):
        return 1j * self.KZ * a

    def dy(self, a):
        return cheb_deriv(a)

    def fields(self, ahat):
        """Physical values and gradient of a spectral vector field: (3,...), (3,3,...)."""
        val = self.to_phys(ahat)
        grad = np.empty((3, 3) + val.shape[1:])
        for i in range(3):
            grad[i, 0] = self.to_phys(self.dx(ahat[i]))
            grad[i, 1] = self.to_phys(self.dy(ahat[i]))
            grad[i, 2] = self.to_phys(self.dz(ahat[i]))
        return val, grad

    # ---------------------------------------------------------------- Stokes step
    def _factor(self, sigma):
        key = float(sigma)
        if key in self._lu:
            return self._lu[key]
        table = {}
        for ij, (A, scale) in self.stokes_systems(sigma).items():
            table[ij] = sla.lu_factor(A) if scale is None else (sla.lu_factor(A * scale[:, None]), scale)
        self._lu[key] = table
        return table

    def stokes_systems(self, sigma):
        """The dense tau system of every mode: {(i, j): (A, row scale)}; the mean mode's
        real Dirichlet Helmholtz matrix has no scale (None)."""
        N, n1 = self.N, self.N + 1
        I = np.eye(n1)
        D = self.Dmat
        D2 = D @ D
        alt = (-1.0) ** np.arange(n1)
        table = {}
        for i in range(self.Mx):
            for j in range(self.Mz):
                kx, kz = self.kx[i], self.kz[j]
                k2 = kx * kx + kz * kz
                if k2 == 0.0:
                    A = np.zeros((n1, n1))
                    A[: N - 1] = (sigma * I - D2)[: N - 1]
                    A[N - 1] = 1.0
                    A[N] = alt
                    table[(i, j)] = (A, None)
                    continue
                H = (sigma + k2) * I - D2
                grads = [1j * kx * I, D, 1j * kz * I]
                A = np.zeros((4 * n1, 4 * n1), np.complex128)
                r = 0
                for c in range(3):
                    for row in range(N - 1):
                        A[r, c * n1:(c + 1) * n1] = H[row]
                        A[r, 3 * n1:] = grads[c][row]
                        r += 1
                for c in range(3):
                    A[r, c * n1:(c + 1) * n1] = 1.0
                    A[r + 1, c * n1:(c + 1) * n1] = alt
                    r += 2
                for row in range(n1):
                    for c in range(3):
                        A[r, c * n1:(c + 1) * n1] = grads[c][row]
                    r += 1
                scale = 1.0 / np.abs(A).max(axis=1)
                table[(i, j)] = (A, scale)
        return table

    def stokes(self, F, sigma):
        """Solve the tau Stokes problem for every mode; F: right-hand side (3, Mx, Mz, Ny)."""
        table = self._factor(sigma)
        N, n1 = self.N, self.N + 1
        out = np.zeros_like(F, dtype=np.complex128)
        for (i, j), fac in table.items():
            if self.kx[i] == 0.0 and self.kz[j] == 0.0:
                for c in (0, 2):
                    b = np.zeros(n1, np.complex128)
                    b[: N - 1] = F[c, i, j, : N - 1]
                    out[c, i, j] = sla.lu_solve(fac, b)
                continue
            lu, scale = fac
            b = np.zeros(4 * n1, np.complex128)
            for c in range(3):
                b[c * (N - 1):(c + 1) * (N - 1)] = F[c, i, j, : N - 1]
            x = sla.lu_solve(lu, b * scale)
            for c in range(3):
                out[c, i, j] = x[c * n1:(c + 1) * n1]
        return out

    def stokes_step(self, rhs, step):
        """Implicit step of size ``step``: (1/step - nu Lap) w + grad p = rhs, div w = 0, w(+-1) = 0."""
        return self.stokes(rhs / self.nu, 1.0 / (self.nu * step))

    # ---------------------------------------------------------------- method
    def M_hat(self, uval, ugrad):
        return self.to_spec(nonlinear_M(uval, ugrad, self.U_phys, self.dU_phys, self.V_base))

    def N_hat(self, qval, qgrad, uval, ugrad):
        return self.to_spec(adjoint_N(qval, qgrad, uval, ugrad, self.U_phys, self.dU_phys, self.V_base))

    def norm_phys(self, val):
        """Volume-normalised L2 norm of physical values (3, Ny, Nx, Nz)."""
        s = (val ** 2).sum(axis=0).mean(axis=(-2, -1))
        return math.sqrt(0.5 * float((self.w_cc * s).sum()))

    def norm(self, ahat):
        return self.norm_phys(self.to_phys(ahat))

    def residual(self, uhat, return_fields=False):
        """§4 steps 1-2: r1 = (Phi_dt(u) - u)/dt and J = ||r1||."""
        uval, ugrad = self.fields(uhat)
        u_dt = self.stokes_step(uhat / self.dt + self.M_hat(uval, ugrad), self.dt)
        r1 = (u_dt - uhat) / self.dt
        J = self.norm(r1)
        if return_fields:
            return r1, J, (uval, ugrad)
        return r1, J

    def adjoint_direction(self, uhat, r1, ufields=None):
        """§4 steps 3-4: f = -(Psi_dtauhat(r1) - r1)/dtau_hat."""
        uval, ugrad = ufields if ufields is not None else self.fields(uhat)
        qval, qgrad = self.fields(r1)
        Nh = self.N_hat(qval, qgrad, uval, ugrad)
        r1_plus = self.stokes_step(r1 / self.dtau_hat + Nh, self.dtau_hat)
        return -(r1_plus - r1) / self.dtau_hat

    def descent_step(self, uhat, dtau):
        """§4 steps 1-5; returns (u + dtau f, J(u), r1, f)."""
        r1, J, uf = self.residual(uhat, return_fields=True)
        f = self.adjoint_direction(uhat, r1, uf)
        return uhat + dtau * f, J, r1, f

    def run(self, uhat, dtau, nsteps):
        """Repeated descent steps; returns final state and the J history (J before each step)."""
        hist = []
        u = uhat
        for _ in range(nsteps):
            u, J, _, _ = self.descent_step(u, dtau)
            hist.append(J)
        return u, np.array(hist)

    # ---------------------------------------------------------------- symmetries (§5.1)
    def _grid_map(self, a, ix, iy, iz, signs):
        """Field g with g_c(x_i, y_j, z_k) = signs_c * a_c(x_ix[i], y_iy[j], z_iz[k])."""
        val = self.to_phys(a)
        g = val[:, iy][:, :, ix][:, :, :, iz] * np.asarray(signs, float)[:, None, None, None]
        return self.to_spec(g)

    def s1(self, a):
        """s1 [u,v,w](x,y,z) = [-u,-v,w](-x + Lx/2, -y, z + Lz/2) (§5.1).  On the grid:
        x_i -> x at index (nx/2 - i) mod nx, y_j -> y_{N-j}, z_k -> z at (k + nz/2) mod nz."""
        ix = (self.nx // 2 - np.arange(self.nx)) % self.nx
        iy = self.N - np.arange(self.N + 1)
        iz = (np.arange(self.nz) + self.nz // 2) % self.nz
        return self._grid_map(a, ix, iy, iz, (-1.0, -1.0, 1.0))

    def s2(self, a):
        """s2 [u,v,w](x,y,z) = [u,v,-w](x + Lx/2, y, -z) (§5.1)."""
        ix = (np.arange(self.nx) + self.nx // 2) % self.nx
        iy = np.arange(self.N + 1)
        iz = (-np.arange(self.nz)) % self.nz
        return self._grid_map(a, ix, iy, iz, (1.0, 1.0, -1.0))

    def symmetrize(self, a, mask):
        """Group average over the symmetries selected by mask (bit 0: s1, bit 1: s2): the
        projection onto the subspace invariant under all of them."""
        terms = [a]
        if mask & 1:
            terms.append(self.s1(a))
        if mask & 2:
            terms += [self.s2(t) for t in terms]
        return sum(terms) / len(terms)

    # ---------------------------------------------------------------- DNS (§5.2)
    def dns(self, uhat, nsteps):
        """nsteps of u <- u^dt = u + dt r1 (the Stokes step of §4 step 1 as a time stepper).
        Returns the final state and h_s = ||u_s|| for s = 0..nsteps-1 (before each step)."""
        u = uhat
        h = []
        for _ in range(nsteps):
            h.append(self.norm(u))
            r1, _ = self.residual(u)
            u = u + self.dt * r1
        return u, np.array(h)

    @staticmethod
    def extrema(h):
        """Steps s (1 <= s <= len(h) - 2) where h has a strict local extremum."""
        return [s for s in range(1, len(h) - 1) if (h[s] - h[s - 1]) * (h[s + 1] - h[s]) < 0]

    # ---------------------------------------------------------------- checks
    def divergence(self, ahat):
        return self.dx(ahat[0]) + self.dy(ahat[1]) + self.dz(ahat[2])

    def wall_values(self, ahat):
        n = np.arange(self.N + 1)
        return ahat.sum(axis=-1), (ahat * ((-1.0) ** n)).sum(axis=-1)

    # ---------------------------------------------------------------- snapshot vector
    def independent_modes(self):
        """(i, j) storage indices of independent modes (m, p) != (0, 0): p > 0 all m; p = 0, m > 0."""
        out = []
        for i in range(self.Mx):
            for j in range(self.Mz):
                if j > 0 or (1 <= self.m[i]):
                    out.append((i, j))
        return out

    def psi_dim(self):
        N = self.N
        return len(self.independent_modes()) * (2 * (N - 3) + 2 * (N - 1)) + 2 * (N - 1)

    def to_psi(self, uhat):
        """Minimal real coordinates of an admissible field (§6.2): free coefficients of
        v (0..N-4) and wall-normal vorticity eta = i kz u - i kx w (0..N-2) per independent
        mode (real and imaginary parts), and the mean u, w (0..N-2)."""
        N = self.N
        parts = []
        for (i, j) in self.independent_modes():
            v = uhat[1, i, j, : N - 3]
            eta = (1j * self.kz[j] * uhat[0, i, j] - 1j * self.kx[i] * uhat[2, i, j])[: N - 1]
            parts += [v.real, v.imag, eta.real, eta.imag]
        parts += [uhat[0, 0, 0, : N - 1].real, uhat[2, 0, 0, : N - 1].real]
        return np.concatenate(parts)

    def from_psi(self, psi):
        """Inverse of ``to_psi``: complete the wall conditions and rebuild (u, v, w)."""
        N, n1 = self.N, self.N + 1
        n = np.arange(n1)
        alt = (-1.0) ** n
        # wall-condition rows: value(+1), value(-1), slope(+1), slope(-1)
        Bc = np.stack([np.ones(n1), alt, n ** 2.0, -alt * n ** 2.0])
        Bd = np.stack([np.ones(n1), alt])
        out = np.zeros((3, self.Mx, self.Mz, n1), np.complex128)
        pos = 0

        def take(L):
            nonlocal pos
            seg = psi[pos:pos + L]
            pos += L
            return seg
        for (i, j) in self.independent_modes():
            v = np.zeros(n1, np.complex128)
            eta = np.zeros(n1, np.complex128)
            v[: N - 3] = take(N - 3) + 1j * take(N - 3)
            eta[: N - 1] = take(N - 1) + 1j * take(N - 1)
            v[N - 3:] = np.linalg.solve(Bc[:, N - 3:], -Bc[:, : N - 3] @ v[: N - 3])
            eta[N - 1:] = np.linalg.solve(Bd[:, N - 1:], -Bd[:, : N - 1] @ eta[: N - 1])
            kx, kz = self.kx[i], self.kz[j]
            k2 = kx * kx + kz * kz
            xi = -cheb_deriv(v)
            out[0, i, j] = (-1j * kx * xi - 1j * kz * eta) / k2
            out[1, i, j] = v
            out[2, i, j] = (-1j * kz * xi + 1j * kx * eta) / k2
            if j == 0:
                out[:, self.Mx - i, 0] = np.conj(out[:, i, 0])
        for c in (0, 2):
            a = np.zeros(n1)
            a[: N - 1] = take(N - 1)
            a[N - 1:] = np.linalg.solve(Bd[:, N - 1:], -Bd[:, : N - 1] @ a[: N - 1])
            out[c, 0, 0] = a
        assert pos == len(psi)
        return out
