"""Seeded synthetic initial guesses for plane Couette flow (shared by the oracle and the CUDA path).

This module holds no step of the adjoint-descent method.  It only builds admissible
initial velocity perturbations (divergence-free, zero at the walls) in the
Fourier(x) x Chebyshev(y) x Fourier(z) coefficient layout that both the oracle and the
CUDA library consume.  It carries its own small Chebyshev helpers (derivative, boundary
completion, exact L2 Gram integral) so that it imports nothing from either side.

Spectral layout (paper §4, Eq. (Foureir_Chebyshev_Fourier)): complex128 array
``[3][Mx][Mz][Ny]`` (component, x-mode, z-mode, Chebyshev index), with Ny fastest.
x-modes are stored m = 0..Kx, -Kx..-1 (Mx = 2Kx+1); z-modes p = 0..Kz (Mz = Kz+1),
the p<0 half being the complex conjugate (real fields).  Kx = Nx//3 - 1,
Kz = Nz//3 - 1 (2/3 dealiasing; the only choice that reproduces the paper's snapshot
dimension N = 20218 at 32x31x32, §6.2).

Recipes (synthetic stand-ins for the paper's DNS snapshots, §5.1):
* ``random_perturbation``: per mode, v = (1-y^2)^2 sum a_n T_n and wall-normal
  vorticity eta = (1-y^2) sum b_n T_n with coefficient variance proportional to
  exp(-|(m, p, n)|); converted to (u, v, w) with the divergence constraint; mean
  (m = p = 0) u, w = (1-y^2) sum c_n T_n; rescaled to an exact L2 norm.
* ``streak_roll``: streamwise-independent rolls (v at (m, p) = (0, 1)), a streak
  (eta at (0, 1)) whose wavy x-modulation sits at (+-1, 1), random phases per seed,
  plus a ``random_perturbation`` noise field.
"""
import math

import numpy as np

TWO_PI = 2.0 * math.pi
LX_PAPER = TWO_PI / 1.14
LZ_PAPER = TWO_PI / 2.5


def mode_layout(nx, ny, nz):
    """Return (Kx, Kz, Mx, Mz, N, m_of_index, p_of_index) for a grid Nx x Ny x Nz."""
    Kx = nx // 3 - 1
    Kz = nz // 3 - 1
    Mx = 2 * Kx + 1
    Mz = Kz + 1
    m = np.array(list(range(0, Kx + 1)) + list(range(-Kx, 0)), dtype=np.int64)
    p = np.arange(Mz, dtype=np.int64)
    return Kx, Kz, Mx, Mz, ny - 1, m, p


def _cheb_diff(a):
    """Coefficients of d/dy of a Chebyshev series (last axis)."""
    N = a.shape[-1] - 1
    b = np.zeros_like(a)
    if N >= 1:
        b[..., N - 1] = 2 * N * a[..., N]
    for n in range(N - 2, -1, -1):
        b[..., n] = b[..., n + 2] + 2 * (n + 1) * a[..., n + 1]
    b[..., 0] *= 0.5
    return b


def _cheb_mul(a, c):
    """Chebyshev series product a(y) * c(y) with c of low degree; result truncated to len(a)."""
    L = a.shape[-1]
    out = np.zeros(a.shape[:-1] + (L + len(c),), dtype=np.result_type(a, np.float64))
    for j, cj in enumerate(c):
        if cj == 0.0:
            continue
        for i in range(L):
            out[..., i + j] += 0.5 * cj * a[..., i]
            out[..., abs(i - j)] += 0.5 * cj * a[..., i]
    return out[..., :L]


# (1 - y^2) and (1 - y^2)^2 as Chebyshev series
WALL1 = [0.5, 0.0, -0.5]
WALL2 = [0.375, 0.0, -0.5, 0.0, 0.125]


def _complete_dirichlet(a):
    """Return (1 - y^2) * a(y), keeping the degree <= N (a's top two coefficients dropped)."""
    b = a.copy()
    b[..., -2:] = 0
    return _cheb_mul(b, WALL1)


def _complete_clamped(a):
    """Return (1 - y^2)^2 * a(y), keeping the degree <= N (a's top four coefficients dropped)."""
    b = a.copy()
    b[..., -4:] = 0
    return _cheb_mul(b, WALL2)


def _gram(N):
    """Exact integral over [-1, 1] of T_a T_b."""
    a = np.arange(N + 1)
    s = a[:, None] + a[None, :]
    d = np.abs(a[:, None] - a[None, :])

    def h(j):
        out = np.zeros(j.shape)
        even = j % 2 == 0
        out[even] = 1.0 / (1.0 - j[even].astype(float) ** 2)
        return out
    return h(s) + h(d)


def exact_l2(uhat):
    """Volume-normalised L2 norm sqrt((1/(2 Lx Lz)) int |u|^2) of a spectral field (exact)."""
    N = uhat.shape[-1] - 1
    G = _gram(N)
    Mz = uhat.shape[-2]
    wp = np.where(np.arange(Mz) == 0, 1.0, 2.0)
    quad = np.einsum("...n,nk,...k->...", uhat.conj(), G, uhat).real
    return math.sqrt(0.5 * float((quad * wp[None, None, :]).sum()))


def _assemble(v, eta, umean, wmean, nx, nz, Lx, Lz):
    """(v, eta) per mode + mean (u, w) -> (u, v, w) coefficients, divergence-free."""
    Kx, Kz, Mx, Mz, N, m, p = mode_layout(nx, 0, nz)
    kx = TWO_PI * m / Lx
    kz = TWO_PI * p / Lz
    KX = kx[:, None, None]
    KZ = kz[None, :, None]
    k2 = KX ** 2 + KZ ** 2
    k2s = np.where(k2 == 0, 1.0, k2)
    xi = -_cheb_diff(v)                  # i kx u + i kz w = -dv/dy
    u = (-1j * KX * xi - 1j * KZ * eta) / k2s
    w = (-1j * KZ * xi + 1j * KX * eta) / k2s
    out = np.stack([u, v, w]).astype(np.complex128)
    out[:, 0, 0, :] = 0
    out[0, 0, 0, :] = umean
    out[2, 0, 0, :] = wmean
    return out


def _hermitian_p0(a, Kx):
    """Make the p = 0 plane conjugate-symmetric in m (real physical field)."""
    Mx = 2 * Kx + 1
    for i in range(1, Kx + 1):
        a[..., Mx - i, 0, :] = np.conj(a[..., i, 0, :])
    a[..., 0, 0, :] = a[..., 0, 0, :].real
    return a


def random_perturbation(nx, ny, nz, amplitude=0.1, seed=0, Lx=LX_PAPER, Lz=LZ_PAPER):
    """Divergence-free, no-slip random field with coefficient variance ~ exp(-|(m,p,n)|)."""
    Kx, Kz, Mx, Mz, N, m, p = mode_layout(nx, ny, nz)
    rng = np.random.Generator(np.random.Philox(seed))
    n = np.arange(N + 1)
    kap = np.sqrt(m[:, None, None] ** 2 + p[None, :, None] ** 2 + n[None, None, :] ** 2)
    sd = np.exp(-0.5 * kap)

    def draw():
        return sd * (rng.standard_normal(sd.shape) + 1j * rng.standard_normal(sd.shape))
    v = _complete_clamped(draw())
    eta = _complete_dirichlet(draw())
    v = _hermitian_p0(v, Kx)
    eta = _hermitian_p0(eta, Kx)
    um = _complete_dirichlet(sd[0, 0] * rng.standard_normal(N + 1))
    wm = _complete_dirichlet(sd[0, 0] * rng.standard_normal(N + 1))
    u = _assemble(v, eta, um, wm, nx, nz, Lx, Lz)
    u = _hermitian_p0(u, Kx)
    s = exact_l2(u)
    return u * (amplitude / s) if s > 0 else u


def _profile_clamped(N, coeffs):
    a = np.zeros(N + 1)
    a[: len(coeffs)] = coeffs
    return _complete_clamped(a)


def _profile_dirichlet(N, coeffs):
    a = np.zeros(N + 1)
    a[: len(coeffs)] = coeffs
    return _complete_dirichlet(a)


def streak_roll(nx, ny, nz, seed=0, roll=0.05, streak=0.1, noise=0.02, Lx=LX_PAPER, Lz=LZ_PAPER):
    """Rolls (0,1) + wavy streak ((0,1) and (+-1,1)) + random noise, all no-slip and div-free."""
    Kx, Kz, Mx, Mz, N, m, p = mode_layout(nx, ny, nz)
    rng = np.random.Generator(np.random.Philox(10_000 + seed))
    ph = rng.uniform(0, TWO_PI, size=3)
    zero = np.zeros((Mx, Mz, N + 1), np.complex128)
    # rolls: v = (1 - y^2)^2 cos(beta z + phi0)
    v = zero.copy()
    v[0, 1] = 0.5 * np.exp(1j * ph[0]) * _profile_clamped(N, [1.0])
    rolls = _assemble(v, zero.copy(), np.zeros(N + 1), np.zeros(N + 1), nx, nz, Lx, Lz)
    rolls *= roll / exact_l2(rolls)
    # streak: eta = du/dz - dw/dx with profile (1 - y^2) y; wavy modulation at m = +-1
    eta = zero.copy()
    prof = _profile_dirichlet(N, [0.0, 1.0])
    eta[0, 1] = 0.5 * np.exp(1j * ph[1]) * prof
    eta[1, 1] = 0.25 * np.exp(1j * ph[2]) * prof
    eta[Mx - 1, 1] = 0.25 * np.exp(-1j * ph[2]) * prof
    streaks = _assemble(zero.copy(), eta, np.zeros(N + 1), np.zeros(N + 1), nx, nz, Lx, Lz)
    streaks *= streak / exact_l2(streaks)
    out = rolls + streaks + random_perturbation(nx, ny, nz, noise, seed, Lx, Lz)
    return _hermitian_p0(out, Kx)


def batch(generator, seeds, *args, **kw):
    """Stack ``generator(*args, seed=s, **kw)`` over seeds -> [B][3][Mx][Mz][Ny]."""
    return np.stack([generator(*args, seed=s, **kw) for s in seeds])
