"""Pins of the FP64 oracle against what the paper and mathematics fix (CPU only).

Each test compares the oracle with something other than itself: closed forms,
exact quadrature, manufactured solutions built with numpy's Chebyshev routines,
symmetries the paper states, and the adjoint identity of its Appendix A.
"""
import math

import numpy as np
import pytest
from numpy.polynomial import chebyshev as npC

import pcf_inputs as gi
from oracle import PCFOracle, dmd
from oracle import pcf_oracle as po
from tests.analytic_fields import Grid, Scalar, vector_eval
from tests.paper_values import paper_values

LX, LZ = gi.LX_PAPER, gi.LZ_PAPER


@pytest.fixture(scope="module")
def o16():
    return PCFOracle(16, 17, 16)


# ------------------------------------------------------------------ transforms
@pytest.mark.parametrize("N", [8, 16, 32, 96])
def test_cheb_derivative_exact(N):
    """d/dy T_n = n U_{n-1}(y) = n sin(n t)/sin(t), y = cos t, for every n <= N."""
    t = np.linspace(0.1, 3.0, 23)
    y = np.cos(t)
    for n in range(N + 1):
        e = np.zeros(N + 1)
        e[n] = 1.0
        got = npC.chebval(y, po.cheb_deriv(e))
        want = n * np.sin(n * t) / np.sin(t)
        assert np.max(np.abs(got - want)) <= 1e-13 * max(1, n * n)


@pytest.mark.parametrize("N", [16, 32, 48, 96])
def test_clenshaw_curtis_exact(N):
    """sum_j w_j T_n(y_j) = int T_n = 2/(1-n^2) (n even), 0 (n odd), for n <= N."""
    w = po.clenshaw_curtis_weights(N)
    y = np.cos(math.pi * np.arange(N + 1) / N)
    for n in range(N + 1):
        want = 2.0 / (1.0 - n * n) if n % 2 == 0 else 0.0
        assert abs((w * np.cos(n * np.arccos(y))).sum() - want) <= 1e-14 * N


def test_single_mode_synthesis(o16):
    """A single (m, p, n) coefficient synthesises to 2 Re(c T_n(y) e^{i(kx x + kz z)})."""
    rng = np.random.default_rng(1)
    x = np.arange(o16.nx) * LX / o16.nx
    z = np.arange(o16.nz) * LZ / o16.nz
    for (i, j, n) in [(1, 1, 3), (o16.Mx - 2, 2, 7), (2, 0, 0), (0, 3, 16)]:
        a = np.zeros((o16.Mx, o16.Mz, o16.N + 1), np.complex128)
        c = rng.standard_normal() + 1j * rng.standard_normal()
        a[i, j, n] = c
        if j == 0:
            a[o16.Mx - i, 0, n] = np.conj(c)
        got = o16.to_phys(a)
        kx, kz = o16.kx[i], o16.kz[j]
        E = np.exp(1j * (kx * x[:, None] + kz * z[None, :]))
        Tn = np.cos(n * np.arccos(o16.y))[:, None, None]
        want = 2 * np.real(c * E)[None] * Tn
        assert np.max(np.abs(got - want)) < 1e-13


def test_round_trip(o16):
    u = gi.random_perturbation(16, 17, 16, 0.1, 3)
    assert np.max(np.abs(o16.to_spec(o16.to_phys(u)) - u)) < 1e-15


# ------------------------------------------------------------------ Stokes step
def _manufactured(o, sigma, rng):
    """Admissible (u, v, w) plus arbitrary P; F = (sigma - Lap) u + grad P via numpy Chebyshev."""
    u = gi.random_perturbation(o.nx, o.ny, o.nz, 1.0, int(rng.integers(1 << 30)))
    P = rng.standard_normal(u.shape[1:]) + 1j * rng.standard_normal(u.shape[1:])
    P[0, 0] = 0.0
    F = np.zeros_like(u)
    for i in range(o.Mx):
        for j in range(o.Mz):
            kx, kz = o.kx[i], o.kz[j]
            k2 = kx * kx + kz * kz
            for c in range(3):
                prof = u[c, i, j]
                lap = np.zeros(o.N + 1, np.complex128)
                d2 = npC.chebder(prof, 2)
                lap[: len(d2)] = d2
                F[c, i, j] = (sigma + k2) * prof - lap
            F[0, i, j] += 1j * kx * P[i, j]
            F[2, i, j] += 1j * kz * P[i, j]
            dP = npC.chebder(P[i, j])
            F[1, i, j, : len(dP)] += dP
    return u, F


@pytest.mark.parametrize("grid", [(16, 17, 16), (32, 33, 32)])
def test_stokes_manufactured(grid):
    """The tau Stokes solve recovers an admissible polynomial field exactly."""
    o = PCFOracle(*grid)
    rng = np.random.default_rng(7)
    sigma = 1.0 / (o.nu * o.dt)
    u, F = _manufactured(o, sigma, rng)
    got = o.stokes(F, sigma)
    assert np.max(np.abs(got - u)) <= 1e-12 * np.max(np.abs(u)) * 100


def test_stokes_output_admissible(o16):
    """Any right-hand side gives a divergence-free (all coefficients), no-slip output."""
    rng = np.random.default_rng(2)
    F = rng.standard_normal((3, o16.Mx, o16.Mz, o16.N + 1)) + 1j * rng.standard_normal((3, o16.Mx, o16.Mz, o16.N + 1))
    F[:, o16.Mx - 1:o16.Kx:-1, 0] = np.conj(F[:, 1:o16.Kx + 1, 0])
    out = o16.stokes_step(F, 0.25)
    scale = np.max(np.abs(out))
    assert np.max(np.abs(o16.divergence(out))) <= 1e-12 * scale * 10
    for wv in o16.wall_values(out):
        assert np.max(np.abs(wv)) <= 1e-12 * scale


# ------------------------------------------------------------------ the method
def test_laminar_is_equilibrium(o16):
    """u = 0 (laminar Couette u_b = y) gives r1 = 0 and f = 0 exactly (§5)."""
    z = np.zeros((3, o16.Mx, o16.Mz, o16.N + 1), np.complex128)
    r1, J = o16.residual(z)
    assert J == 0.0 and np.all(r1 == 0)
    assert np.all(o16.adjoint_direction(z, r1) == 0)


@pytest.mark.parametrize("base", ["poiseuille", "asbl"])
def test_laminar_is_equilibrium_for_other_base_flows(base):
    """u = 0 is an equilibrium for the plane Poiseuille and suction boundary layer base flows
    too: r1 = f = 0 exactly."""
    o = PCFOracle(16, 17, 16, base_flow=base, suction_length=0.5 if base == "asbl" else None)
    z = np.zeros((3, o.Mx, o.Mz, o.N + 1), np.complex128)
    r1, J = o.residual(z)
    assert J == 0.0 and np.all(r1 == 0)
    assert np.all(o.adjoint_direction(z, r1) == 0)


def _mirror_y(o, a):
    """[u,v,w](x,y,z) -> [u,-v,w](x,-y,z): T_n(-y) = (-1)^n T_n(y)."""
    sgn = (-1.0) ** np.arange(o.N + 1)
    out = a * sgn
    out[1] = -out[1]
    return out


@pytest.mark.parametrize("base,symmetric", [("poiseuille", True), ("couette", False), ("asbl", False)])
def test_mirror_symmetry_of_the_base_flow(base, symmetric):
    """U = 1 - y^2 is even in y, so the Poiseuille descent commutes with the y mirror; the
    odd Couette profile U = y breaks it, and so does the suction boundary layer (one-sided
    profile, suction V != 0): the test tells the base flows apart."""
    o = PCFOracle(16, 17, 16, base_flow=base, suction_length=0.5 if base == "asbl" else None)
    u = gi.random_perturbation(16, 17, 16, 0.1, 4)
    a1 = _mirror_y(o, o.descent_step(u, 0.01)[0])
    a2 = o.descent_step(_mirror_y(o, u), 0.01)[0]
    err = np.max(np.abs(a1 - a2)) / np.max(np.abs(a1))
    assert (err <= 1e-13) if symmetric else (err > 1e-6)


def test_r1_and_f_admissible(o16):
    """§4 steps 2 and 4: r1 and f are divergence-free and vanish at the walls."""
    u = gi.random_perturbation(16, 17, 16, 0.1, 0)
    _, _, r1, f = o16.descent_step(u, 0.01)
    for a in (r1, f):
        scale = np.max(np.abs(a))
        assert np.max(np.abs(o16.divergence(a))) <= 1e-13 * scale * 100
        for wv in o16.wall_values(a):
            assert np.max(np.abs(wv)) <= 1e-14 * scale * 100


def _d2(a):
    """Second y-derivative of Chebyshev coefficients (numpy's Chebyshev module), same length."""
    return np.pad(npC.chebder(a, m=2, axis=-1), [(0, 0)] * (a.ndim - 1) + [(0, 2)])


def _step_equation_gap(o, u):
    """Largest relative residual of (I - dt nu Lap) r1 = M(u) + nu Lap u on the Chebyshev rows
    0..N-2, for the wall-normal vorticity i kz r_x - i kx r_z of every mode (no pressure) and
    for r_x, r_z of the mean mode (no mean pressure gradient).  M is the unmodified oracle's,
    so a mistake planted in the residual path shows."""
    r1, _, (uval, ugrad) = o.residual(u, return_fields=True)
    M = PCFOracle.M_hat(o, uval, ugrad)
    k2 = o.KX ** 2 + o.KZ ** 2
    rows = slice(0, o.N - 1)

    def lap(a):
        return _d2(a) - k2 * a

    def eta(a):
        return 1j * o.KZ * a[0] - 1j * o.KX * a[2]

    lhs = eta(r1) - o.dt * o.nu * lap(eta(r1))
    rhs = eta(M) + o.nu * lap(eta(u))
    gap = np.abs(lhs - rhs)[..., rows].max() / np.abs(rhs[..., rows]).max()
    for c in (0, 2):
        lm = r1[c, 0, 0] - o.dt * o.nu * _d2(r1[c, 0, 0])
        rm = M[c, 0, 0] + o.nu * _d2(u[c, 0, 0])
        gap = max(gap, np.abs(lm - rm)[rows].max() / np.abs(rm[rows]).max())
    return gap


@pytest.mark.parametrize("dt", [0.05, 0.25, 1.0])
def test_r1_solves_the_step_equation_for_every_dt(dt):
    """§4 steps 1-2: u^dt = u + dt r1 solves (1/dt - nu Lap) u^dt + grad p = u/dt + M(u), so
    (I - dt nu Lap) r1 + grad p = M(u) + nu Lap u.  The right-hand side does not depend on dt:
    r1 = 0 exactly where u is an equilibrium of the discrete equations, whatever the step
    (§4).  Checked where pressure drops out, on the rows where the momentum equations hold
    (the last two rows of each field carry the no-slip conditions instead)."""
    u = gi.random_perturbation(16, 17, 16, 0.1, 3)
    assert _step_equation_gap(PCFOracle(16, 17, 16, dt=dt), u) <= 1e-12


class _ViscosityDropped(PCFOracle):
    def stokes_step(self, rhs, step):       # shift 1/step instead of 1/(nu step)
        return self.stokes(rhs / self.nu, 1.0 / step)


class _QuotientWithoutDt(PCFOracle):
    def residual(self, uhat, return_fields=False):
        r1, J, f = PCFOracle.residual(self, uhat, return_fields=True)
        return (r1 * self.dt, J, f) if return_fields else (r1 * self.dt, J)


class _ProductSignFlipped(PCFOracle):
    def M_hat(self, uval, ugrad):
        return -PCFOracle.M_hat(self, uval, ugrad)


@pytest.mark.parametrize("bad", [_ViscosityDropped, _QuotientWithoutDt, _ProductSignFlipped])
def test_step_equation_catches_planted_mistakes(bad):
    """A wrong implicit shift, a missing 1/dt in the quotient or a flipped explicit term
    breaks the step equation by many orders of magnitude."""
    u = gi.random_perturbation(16, 17, 16, 0.1, 3)
    assert _step_equation_gap(bad(16, 17, 16, dt=0.25), u) > 1e-4


def _adjoint_step_gap(o, u):
    """Largest relative residual of (I - dtau_hat nu Lap) f = -(N(r1) + nu Lap r1) (up to a
    gradient) on the momentum rows, for the wall-normal vorticity and the mean mode's x, z
    components.  N is the unmodified oracle's."""
    r1, _, uf = PCFOracle.residual(o, u, return_fields=True)
    f = o.adjoint_direction(u, r1, uf)
    qval, qgrad = PCFOracle.fields(o, r1)
    Nh = PCFOracle.N_hat(o, qval, qgrad, *uf)
    k2 = o.KX ** 2 + o.KZ ** 2
    rows, h = slice(0, o.N - 1), o.dtau_hat * o.nu

    def lap(a):
        return _d2(a) - k2 * a

    def eta(a):
        return 1j * o.KZ * a[0] - 1j * o.KX * a[2]

    lhs = eta(f) - h * lap(eta(f))
    rhs = -(eta(Nh) + o.nu * lap(eta(r1)))
    gap = np.abs(lhs - rhs)[..., rows].max() / np.abs(rhs[..., rows]).max()
    for c in (0, 2):
        lm = f[c, 0, 0] - h * _d2(f[c, 0, 0])
        rm = -(Nh[c, 0, 0] + o.nu * _d2(r1[c, 0, 0]))
        gap = max(gap, np.abs(lm - rm)[rows].max() / np.abs(rm[rows]).max())
    return gap


@pytest.mark.parametrize("dtau_hat", [0.02, 0.1, 0.5])
def test_f_solves_the_dummy_step_equation(dtau_hat):
    """§4 steps 3-4: r1^+ solves (1/dtau_hat - nu Lap) r1^+ + grad phi = r1/dtau_hat + N(r1)
    and f = -(r1^+ - r1)/dtau_hat, so (I - dtau_hat nu Lap) f = -(N(r1) + nu Lap r1) up to a
    gradient.  As dtau_hat -> 0 this is the adjoint evolution of §3 (Eq.
    adjoint_evolution_divergence_free) with the sign reading of step 4.  dt = 0.25 differs
    from every dtau_hat here, so the two step sizes cannot be swapped unnoticed."""
    u = gi.random_perturbation(16, 17, 16, 0.1, 5)
    assert _adjoint_step_gap(PCFOracle(16, 17, 16, dt=0.25, dtau_hat=dtau_hat), u) <= 1e-12


class _DirectionSignFlipped(PCFOracle):
    def adjoint_direction(self, uhat, r1, ufields=None):
        return -PCFOracle.adjoint_direction(self, uhat, r1, ufields)


class _DummyStepTakesDt(PCFOracle):
    def adjoint_direction(self, uhat, r1, ufields=None):
        uval, ugrad = ufields if ufields is not None else self.fields(uhat)
        qval, qgrad = self.fields(r1)
        Nh = self.N_hat(qval, qgrad, uval, ugrad)
        r1_plus = self.stokes_step(r1 / self.dtau_hat + Nh, self.dt)    # dt for dtau_hat
        return -(r1_plus - r1) / self.dtau_hat


class _AdjointTermFlipped(PCFOracle):
    def N_hat(self, qval, qgrad, uval, ugrad):
        return -PCFOracle.N_hat(self, qval, qgrad, uval, ugrad)


@pytest.mark.parametrize("bad", [_DirectionSignFlipped, _DummyStepTakesDt, _AdjointTermFlipped])
def test_dummy_step_equation_catches_planted_mistakes(bad):
    """A flipped descent direction, the NSE step size in the dummy step or a flipped adjoint
    term breaks the equation by many orders of magnitude."""
    u = gi.random_perturbation(16, 17, 16, 0.1, 5)
    assert _adjoint_step_gap(bad(16, 17, 16, dt=0.25, dtau_hat=0.1), u) > 1e-4


def test_descent_monotone(o16):
    """J decreases monotonically along the descent for a small step (§2, §3.4)."""
    u = gi.random_perturbation(16, 17, 16, 0.1, 1)
    _, hist = o16.run(u, 0.01, 40)
    assert np.all(np.diff(hist) < 0)


def test_descent_with_the_papers_step_sizes():
    """The paper's test case (§5.1: Re, box, 32 x 31 x 32, dt = dtau_hat = 0.25, dtau = 0.03)
    descends: J falls at every step.  The dummy-dynamics step taken in the diffusive direction
    keeps the forward-Euler update stable at the paper's dtau; an ascent (f with the wrong
    sign) raises J."""
    pv = paper_values()
    o = PCFOracle(pv["nx"], pv["ny"], pv["nz"], Lx=2 * math.pi / pv["Lx_over_2pi_inverse"],
                  Lz=2 * math.pi / pv["Lz_over_2pi_inverse"], Re=pv["Re"], dt=pv["dt"], dtau_hat=pv["dtau_hat"])
    u = gi.streak_roll(pv["nx"], pv["ny"], pv["nz"], seed=3)
    _, hist = o.run(u, pv["dtau"], 12)
    assert np.all(np.diff(hist) < 0)
    _, up = o.run(u, -pv["dtau"], 3)
    assert np.all(np.diff(up) > 0)


def _shift(o, a, lx, lz):
    return a * np.exp(1j * (o.KX * lx + o.KZ * lz))


def _sigma1(o, a):
    """[u,v,w](x,y,z) -> [-u,-v,w](-x,-y,z)."""
    n = np.arange(o.N + 1)
    idx = (-np.arange(o.Mx)) % o.Mx
    out = a[:, idx] * ((-1.0) ** n)
    out[0] *= -1
    out[1] *= -1
    return out


def _sigma2(o, a):
    """[u,v,w](x,y,z) -> [u,v,-w](x,y,-z)."""
    idx = (-np.arange(o.Mx)) % o.Mx
    out = np.conj(a[:, idx])
    out[2] *= -1
    return out


@pytest.mark.parametrize("op", ["shift", "sigma1", "sigma2", "s1"])
def test_equivariance(o16, op):
    """The descent step commutes with the symmetries of plane Couette flow (§3.4, §5)."""
    u = gi.random_perturbation(16, 17, 16, 0.1, 5)
    if op == "shift":
        g = lambda a: _shift(o16, a, 0.37 * LX, 0.81 * LZ)
    elif op == "sigma1":
        g = lambda a: _sigma1(o16, a)
    elif op == "sigma2":
        g = lambda a: _sigma2(o16, a)
    else:
        g = lambda a: _shift(o16, _sigma1(o16, a), LX / 2, LZ / 2)
    a1 = g(o16.descent_step(u, 0.01)[0])
    a2 = o16.descent_step(g(u), 0.01)[0]
    assert np.max(np.abs(a1 - a2)) <= 1e-14


# ------------------------------------------------------------------ continuous pins
BASES = ["couette", "poiseuille", "asbl"]
NU_PIN, DELTA_PIN = 1.0 / 400.0, 0.5   # viscosity of the pins; suction length of the ASBL profile


def _profile(base, nu=NU_PIN):
    """M and N of the oracle for the base flow `base`, as functions of (..., Y)."""
    prof = lambda Y: po.base_profile(base, Y, nu, DELTA_PIN)  # noqa: E731
    M = lambda u, gu, Y: po.nonlinear_M(u, gu, *prof(Y))  # noqa: E731
    N = lambda q, gq, u, gu, Y: po.adjoint_N(q, gq, u, gu, *prof(Y))  # noqa: E731
    return M, N


def _residual(v, gv, lapv, gq, Y, nu, M=po.nonlinear_M):
    """R(U) = [F(v, q), div v], F = M(v) - grad q + nu Lap v (§3.1, Eq. (momentum))."""
    r1 = M(v, gv, Y) - gq + nu * lapv
    r2 = gv[0, 0] + gv[1, 1] + gv[2, 2]
    return r1, r2


def _adjoint(v, gv, r1, gr1, lapr1, rho, grho, Y, nu, Nfun=po.adjoint_N):
    """L+(U; R) of §3.3 / Appendix A: [N(r1) + (div v) r1 + nu Lap r1 - grad rho, div r1]."""
    divv = gv[0, 0] + gv[1, 1] + gv[2, 2]
    a1 = Nfun(r1, gr1, v, gv, Y) + divv[None] * r1 + nu * lapr1 - grho
    a2 = gr1[0, 0] + gr1[1, 1] + gr1[2, 2]
    return a1, a2


def _fields(rng, K, n0, walls):
    return [Scalar.random(rng, K, n0, w, LX, LZ) for w in walls]


def _eval_U(comps, g):
    v, gv, lapv = vector_eval(comps[:3], g)
    q = comps[3].eval(g)
    return v, gv, lapv, np.stack([q["fx"], q["fy"], q["fz"]]), q["f"]


def _adjoint_identity_gap(Nfun=po.adjoint_N, M=po.nonlinear_M):
    rng = np.random.default_rng(11)
    g = Grid(LX, LZ, nf=12, ng=24)
    nu = 1.0 / 400.0
    K, n0 = 1, 5
    U = _fields(rng, K, n0, [1, 1, 1, 0])
    Rf = _fields(rng, K, n0, [1, 1, 1, 0])
    G = _fields(rng, K, n0, [1, 1, 1, 0])
    Up = [a + b for a, b in zip(U, G)]
    Um = [a + b.scaled(-1.0) for a, b in zip(U, G)]
    # L(U; G) = (R(U + G) - R(U - G))/2, exact for the quadratic residual
    vp, gvp, lvp, gqp, _ = _eval_U(Up, g)
    vm, gvm, lvm, gqm, _ = _eval_U(Um, g)
    r1p, r2p = _residual(vp, gvp, lvp, gqp, g.Y, nu, M)
    r1m, r2m = _residual(vm, gvm, lvm, gqm, g.Y, nu, M)
    L1, L2 = 0.5 * (r1p - r1m), 0.5 * (r2p - r2m)
    r, gr, lapr = vector_eval(Rf[:3], g)
    rho = Rf[3].eval(g)
    lhs_t = (L1 * r).sum(axis=0) + L2 * rho["f"]
    v, gv, _, _, _ = _eval_U(U, g)
    a1, a2 = _adjoint(v, gv, r, gr, lapr, rho["f"], np.stack([rho["fx"], rho["fy"], rho["fz"]]), g.Y, nu, Nfun)
    gvv, _, _ = vector_eval(G[:3], g)
    g2 = G[3].eval(g)["f"]
    rhs_t = (gvv * a1).sum(axis=0) + g2 * a2
    lhs, rhs = g.integrate(lhs_t), g.integrate(rhs_t)
    scale = g.integrate(np.abs(lhs_t)) + g.integrate(np.abs(rhs_t))
    return abs(lhs - rhs) / scale


@pytest.mark.parametrize("base", BASES)
def test_adjoint_identity(base):
    """<L(U;G), R> = <G, L+(U;R)> for U, R, G in P0 (Appendix A), exact quadrature; for
    plane Couette (u_b = (y,0,0)) and plane Poiseuille (u_b = (1-y^2,0,0)) base flows."""
    M, N = _profile(base)
    assert _adjoint_identity_gap(Nfun=N, M=M) <= 1e-12


def _bad_N_sign(q, gq, u, gu, y):
    out = po.adjoint_N(q, gq, u, gu, y)
    out[1] = out[1] + 2.0 * q[0]          # flips the sign of the base-flow transpose term
    return out


def _bad_N_index(q, gq, u, gu, y):
    U0 = u[0] + y
    out = np.empty_like(q)
    for i in range(3):
        adv = U0 * gq[i, 0] + u[1] * gq[i, 1] + u[2] * gq[i, 2]
        tr = q[0] * gu[i, 0] + q[1] * gu[i, 1] + q[2] * gu[i, 2]   # (grad U) q instead of (grad U)^T q
        out[i] = adv - tr
    out[1] = out[1] - q[0]
    return out


@pytest.mark.parametrize("bad", [_bad_N_sign, _bad_N_index])
def test_adjoint_identity_catches_planted_mistakes(bad):
    """A dropped or transposed term in N breaks the identity by many orders of magnitude."""
    assert _adjoint_identity_gap(Nfun=bad) > 1e-4


def test_adjoint_identity_catches_a_dropped_suction_term():
    """With suction V = -0.1 (nu = 0.05), an N that advects with u alone instead of u_b + u
    (V dropped from its advection) breaks the identity by eleven orders of magnitude more
    than the quadrature's rounding; the oracle's N keeps it."""
    M, N = _profile("asbl", nu=0.05)

    def no_v(q, gq, u, gu, Y):
        U, dU, _ = po.base_profile("asbl", Y, 0.05, DELTA_PIN)
        return po.adjoint_N(q, gq, u, gu, U, dU, 0.0)

    assert _adjoint_identity_gap(Nfun=N, M=M) <= 1e-12
    assert _adjoint_identity_gap(Nfun=no_v, M=M) > 1e-6


def test_asbl_profile_is_the_laminar_suction_solution():
    """The asymptotic suction boundary layer (named with plane Poiseuille flow in §7): U = 0
    at the suction wall y = -1, uniform suction V < 0, and the profile solves the steady
    x-momentum balance V U' = nu U'' (no pressure gradient); U' is the derivative of U.  The
    derivatives are taken here by Chebyshev interpolation of U's values at 25 points (the
    interpolant's error at delta = 0.5 is below rounding there)."""
    N = 24
    y = np.cos(np.pi * np.arange(N + 1) / N)
    U, dU, V = po.base_profile("asbl", y, NU_PIN, DELTA_PIN)
    c = npC.chebfit(y, U, N)
    d1 = npC.chebval(y, npC.chebder(c))
    d2 = npC.chebval(y, npC.chebder(c, 2))
    assert abs(U[-1]) < 1e-15 and V < 0 and U[0] > 0.98
    assert np.max(np.abs(d1 - dU)) <= 1e-10 * np.max(np.abs(dU))
    assert np.max(np.abs(V * d1 - NU_PIN * d2)) <= 1e-9 * NU_PIN * np.max(np.abs(d2))


def test_asbl_mean_flow_term_is_the_suction_advection():
    """For u = (f(y), 0, 0) every term of M vanishes except the advection by the base flow's
    suction: M = -V f'(y) e_x.  f = 1 - y^2 gives M_x = 2 V y, i.e. the T_1 coefficient 2 V
    of the mean mode, and nothing else."""
    o = PCFOracle(16, 17, 16, base_flow="asbl", suction_length=DELTA_PIN)
    u = np.zeros((3, o.Mx, o.Mz, o.ny), np.complex128)
    u[0, 0, 0, 0], u[0, 0, 0, 2] = 0.5, -0.5          # 1 - y^2 = T_0/2 - T_2/2
    m = o.M_hat(*o.fields(u))
    want = np.zeros_like(m)
    want[0, 0, 0, 1] = 2.0 * o.V_base
    assert o.V_base == -NU_PIN / DELTA_PIN
    assert np.max(np.abs(m - want)) <= 1e-15



_E = lambda Y: np.exp(-(1.0 + Y) / DELTA_PIN)  # noqa: E731


@pytest.mark.parametrize("base,U,dU,V", [
    ("couette", lambda Y: Y, lambda Y: 1.0 + 0.0 * Y, 0.0),
    ("poiseuille", lambda Y: 1.0 - Y * Y, lambda Y: -2.0 * Y, 0.0),
    ("asbl", lambda Y: 1.0 - _E(Y), lambda Y: _E(Y) / DELTA_PIN, -NU_PIN / DELTA_PIN)])
def test_M_is_perturbative_nse(base, U, dU, V):
    """M(u) = -((u_b+u).grad)(u_b+u) + (u_b.grad)u_b with u_b = (U(y), V, 0) (§3.1);
    (u_b.grad)u_b = V U' e_x (zero without suction).  The profile is written out here, not
    taken from the oracle."""
    rng = np.random.default_rng(3)
    g = Grid(LX, LZ, nf=8, ng=10)
    comps = _fields(rng, 1, 4, [1, 1, 1])
    u, gu, _ = vector_eval(comps, g)
    Ut = u.copy()
    Ut[0] += U(g.Y)
    Ut[1] += V
    gUt = gu.copy()
    gUt[0, 1] += dU(g.Y)
    full = -np.einsum("j...,ij...->i...", Ut, gUt)
    full[0] += V * dU(g.Y)
    got = _profile(base)[0](u, gu, g.Y)
    assert np.max(np.abs(got - full)) <= 1e-13


@pytest.mark.parametrize("base", BASES)
def test_gradient_vs_finite_differences(base):
    """dJ^2/dU along G equals 2 <G, L+(U; R(U))> (the gradient of §2), to 1e-6 relative.

    G satisfies g1 = dg1/dy = 0 and g2 = 0 at the walls, so every boundary term of
    Appendix A vanishes for any U in P0 without requiring R(U) in P0.
    """
    M, N = _profile(base)
    rng = np.random.default_rng(5)
    g = Grid(LX, LZ, nf=12, ng=24)
    nu = 1.0 / 400.0
    U = _fields(rng, 1, 5, [1, 1, 1, 0])
    G = _fields(rng, 1, 5, [2, 2, 2, 1])

    def cost(eps):
        comps = []
        for a, b in zip(U, G):
            # promote both to the same wall factor by folding the wall into the coefficients
            comps.append(_sum_fields(a, b, eps))
        v, gv, lv, gq, _ = _eval_U_mixed(comps, g)
        r1, r2 = _residual(v, gv, lv, gq, g.Y, nu, M)
        return g.integrate((r1 ** 2).sum(axis=0) + r2 ** 2)

    eps = 1e-3
    d1 = (cost(eps) - cost(-eps)) / (2 * eps)
    d2 = (cost(eps / 2) - cost(-eps / 2)) / eps
    fd = (4 * d2 - d1) / 3.0        # removes the exact eps^2 term of the quartic
    a_dot = _adjoint_on_residual(U, g, nu, M, N)
    gvv, _, _ = vector_eval(G[:3], g)
    g2 = G[3].eval(g)["f"]
    grad_dot = 2.0 * g.integrate((gvv * a_dot[0]).sum(axis=0) + g2 * a_dot[1])
    assert abs(fd - grad_dot) <= 1e-6 * abs(grad_dot)


class _Mixed:
    """Sum of two Scalars with different wall factors (evaluated term by term)."""

    def __init__(self, parts):
        self.parts = parts

    def eval(self, g):
        evs = [p.eval(g) for p in self.parts]
        return {k: sum(e[k] for e in evs) for k in evs[0]}


def _sum_fields(a, b, eps):
    return _Mixed([a, b.scaled(eps)])


def _eval_U_mixed(comps, g):
    ev = [c.eval(g) for c in comps[:3]]
    v = np.stack([e["f"] for e in ev])
    gv = np.stack([np.stack([e["fx"], e["fy"], e["fz"]]) for e in ev])
    lv = np.stack([e["lap"] for e in ev])
    q = comps[3].eval(g)
    return v, gv, lv, np.stack([q["fx"], q["fy"], q["fz"]]), q["f"]


def _adjoint_on_residual(U, g, nu, M=po.nonlinear_M, Nfun=po.adjoint_N):
    """L+(U; R(U)), with R(U) and its derivatives obtained exactly.

    R(U) is a trigonometric polynomial in (x, z) (degree <= 2K) and a polynomial in y
    (degree well below 40); sampled on an FFT x Chebyshev-Lobatto grid it is interpolated
    exactly (numpy FFT and chebfit), then differentiated and evaluated on the quadrature grid.
    """
    K = U[0].K
    nfx = 4 * K + 8
    ny = 40
    yy = np.cos(np.pi * np.arange(ny + 1) / ny)
    gg = Grid(g.Lx, g.Lz, nf=nfx, ng=2)
    gg.y = yy
    gg.Y = yy[:, None, None]
    v, gv, lv, gq, _ = _eval_U(U, gg)
    r1, r2 = _residual(v, gv, lv, gq, gg.Y, nu, M)

    def spectral(fgrid):
        """Return callables evaluating f, grad f, Lap f on g from samples on gg."""
        Fh = np.fft.fft2(fgrid, axes=(1, 2)) / nfx ** 2
        kx = 2 * np.pi * np.fft.fftfreq(nfx, 1.0 / nfx) / g.Lx
        kz = 2 * np.pi * np.fft.fftfreq(nfx, 1.0 / nfx) / g.Lz
        coef = npC.chebfit(yy, Fh.reshape(ny + 1, -1), ny)      # (ny+1, nfx*nfx)
        X = g.x[None, :, None]
        Z = g.z[None, None, :]
        res = {k: np.zeros((len(g.y), len(g.x), len(g.z))) for k in ("f", "fx", "fy", "fz", "lap")}
        for a in range(nfx):
            for b in range(nfx):
                c = coef[:, a * nfx + b]
                if np.max(np.abs(c)) < 1e-300:
                    continue
                P0 = npC.chebval(g.y, c)[:, None, None]
                P1 = npC.chebval(g.y, npC.chebder(c))[:, None, None]
                P2 = npC.chebval(g.y, npC.chebder(c, 2))[:, None, None]
                E = np.exp(1j * (kx[a] * X + kz[b] * Z))
                res["f"] += np.real(P0 * E)
                res["fx"] += np.real(1j * kx[a] * P0 * E)
                res["fy"] += np.real(P1 * E)
                res["fz"] += np.real(1j * kz[b] * P0 * E)
                res["lap"] += np.real((P2 - (kx[a] ** 2 + kz[b] ** 2) * P0) * E)
        return res
    rr = [spectral(r1[i]) for i in range(3)]
    rh = spectral(r2)
    r = np.stack([e["f"] for e in rr])
    gr = np.stack([np.stack([e["fx"], e["fy"], e["fz"]]) for e in rr])
    lapr = np.stack([e["lap"] for e in rr])
    vq, gvq, _, _, _ = _eval_U(U, g)
    return _adjoint(vq, gvq, r, gr, lapr, rh["f"], np.stack([rh["fx"], rh["fy"], rh["fz"]]), g.Y, nu, Nfun)


# ------------------------------------------------------------------ snapshot vector, DMD
def test_psi_dimension_matches_paper():
    """N = 20218 independent reals at Nx x Ny x Nz = 32 x 31 x 32 (§5.1 grid, §6.2 count)."""
    pv = paper_values()
    assert PCFOracle(pv["nx"], pv["ny"], pv["nz"]).psi_dim() == pv["snapshot_dim"]


@pytest.mark.parametrize("grid", [(16, 17, 16), (32, 33, 32)])
def test_psi_round_trip(grid):
    o = PCFOracle(*grid)
    u = gi.streak_roll(*grid, seed=2)
    psi = o.to_psi(u)
    assert psi.shape == (o.psi_dim(),)
    assert np.max(np.abs(o.from_psi(psi) - u)) < 1e-15


def test_dmd_recovers_affine_fixed_point():
    """Snapshots of psi_{k+1} = psi* + A (psi_k - psi*) with symmetric A, spectrum in (0,1):
    the steady DMD mode is psi* exactly (§6.2: omega_1 = 0, real eigenvalues)."""
    rng = np.random.default_rng(0)
    n, r0, M = 400, 6, 12
    Q, _ = np.linalg.qr(rng.standard_normal((n, r0)))
    mu = np.linspace(0.3, 0.95, r0)
    star = rng.standard_normal(n)
    a = rng.standard_normal(r0)
    S = np.stack([star + Q @ (a * mu ** k) for k in range(M + 1)], axis=1)
    rstar = dmd.snapshot_rank(S, 1e-10)
    assert rstar == r0 + 1
    psi_s, lam = dmd.dmd_steady_state(S, rstar)
    assert abs(lam[0] - 1.0) < 1e-10
    assert np.max(np.abs(psi_s - star)) <= 1e-9 * np.max(np.abs(star))
    best, r, costs = dmd.dmd_extrapolate(S, lambda p: np.linalg.norm(p - star), 1e-10)
    assert r == rstar and costs[r] < 1e-8


# ------------------------------------------------------------------ symmetric subspace (§5.1, §3.4)
def test_symmetries_match_their_spectral_form(o16):
    """The oracle's s1, s2 (applied literally on the collocation grid) equal their
    coefficient-space forms written from the definitions: s1 = shift(Lx/2, Lz/2) sigma1,
    s2 = shift(Lx/2, 0) sigma2."""
    u = gi.random_perturbation(16, 17, 16, 0.1, 11)
    s1 = _shift(o16, _sigma1(o16, u), LX / 2, LZ / 2)
    s2 = _shift(o16, _sigma2(o16, u), LX / 2, 0.0)
    assert np.max(np.abs(o16.s1(u) - s1)) < 1e-16 * 100
    assert np.max(np.abs(o16.s2(u) - s2)) < 1e-16 * 100


def test_symmetry_group(o16):
    """s1 and s2 are commuting involutions, so {e, s1, s2, s1 s2} is a group of order 4 and
    its average is a projection."""
    u = gi.random_perturbation(16, 17, 16, 0.1, 12)
    assert np.max(np.abs(o16.s1(o16.s1(u)) - u)) < 1e-15
    assert np.max(np.abs(o16.s2(o16.s2(u)) - u)) < 1e-15
    assert np.max(np.abs(o16.s1(o16.s2(u)) - o16.s2(o16.s1(u)))) < 1e-15


def _inner(o, a, b):
    return 0.25 * (o.norm(a + b) ** 2 - o.norm(a - b) ** 2)


@pytest.mark.parametrize("mask", [1, 2, 3])
def test_symmetrize_is_an_orthogonal_projection(o16, mask):
    """Idempotent, invariant under each selected symmetry, self-adjoint in the L2 inner
    product of the norm (the symmetries are isometries), and admissible."""
    a = gi.random_perturbation(16, 17, 16, 0.1, 13)
    b = gi.random_perturbation(16, 17, 16, 0.1, 14)
    Pa, Pb = o16.symmetrize(a, mask), o16.symmetrize(b, mask)
    assert np.max(np.abs(o16.symmetrize(Pa, mask) - Pa)) < 1e-16 * 10
    if mask & 1:
        assert np.max(np.abs(o16.s1(Pa) - Pa)) < 1e-16 * 10
    if mask & 2:
        assert np.max(np.abs(o16.s2(Pa) - Pa)) < 1e-16 * 10
    assert abs(_inner(o16, Pa, b) - _inner(o16, a, Pb)) < 1e-14 * o16.norm(a) * o16.norm(b)
    assert 0.1 * o16.norm(a) < o16.norm(Pa) < o16.norm(a)
    lo, hi = o16.wall_values(Pa)
    assert np.max(np.abs(lo)) < 1e-15 and np.max(np.abs(hi)) < 1e-15
    assert np.max(np.abs(o16.divergence(Pa))) < 1e-13


def test_descent_preserves_the_symmetric_subspace(o16):
    """§5.1: a guess symmetric under s1 and s2 stays symmetric along the descent without the
    symmetries being enforced (§3.4: the descent is equivariant under them)."""
    u = o16.symmetrize(gi.random_perturbation(16, 17, 16, 0.1, 15), 3)
    uT, hist = o16.run(u, 0.01, 20)
    assert hist[-1] < hist[0]
    assert np.max(np.abs(o16.symmetrize(uT, 3) - uT)) < 1e-14 * np.max(np.abs(uT))


@pytest.mark.parametrize("base", ["poiseuille", "asbl"])
def test_s1_is_not_a_symmetry_of_poiseuille_flow(base):
    """s1 turns U = 1 - y^2 into -(1 - y^2) (and the suction profile into a blowing one): it
    maps these flows to other flows, so the descent there is not s1-equivariant; s2 leaves
    U(y) and V alone and still is."""
    o = PCFOracle(16, 17, 16, base_flow=base, suction_length=0.5 if base == "asbl" else None)
    u = gi.random_perturbation(16, 17, 16, 0.1, 16)
    gap1 = np.max(np.abs(o.s1(o.descent_step(u, 0.01)[0]) - o.descent_step(o.s1(u), 0.01)[0]))
    gap2 = np.max(np.abs(o.s2(o.descent_step(u, 0.01)[0]) - o.descent_step(o.s2(u), 0.01)[0]))
    assert gap1 > 1e-6 and gap2 < 1e-14


# ------------------------------------------------------------------ DNS with the Stokes step (§5.2)
def test_dns_of_a_mean_flow_perturbation_is_the_implicit_heat_step():
    """For u = (f(y), 0, 0) all terms of M vanish and the Stokes step is implicit Euler for
    df/dt = nu f''.  f = cos(pi y / 2) is the slowest Dirichlet mode, so each DNS step
    multiplies it by 1 / (1 + nu dt pi^2 / 4) (to the tau method's spectral accuracy)."""
    o = PCFOracle(16, 17, 16, dt=0.05)
    u = np.zeros((3, o.Mx, o.Mz, o.ny), np.complex128)
    u[0, 0, 0] = o.Cinv @ np.cos(0.5 * math.pi * o.y)
    u[2, 0, 0] = -0.5 * u[0, 0, 0]
    uT, h = o.dns(u, 8)
    g = 1.0 / (1.0 + o.nu * o.dt * math.pi ** 2 / 4)
    assert np.max(np.abs(uT - g ** 8 * u)) < 1e-13
    assert np.allclose(h[1:] / h[:-1], g, rtol=0, atol=1e-13)


def test_extrema_brute_force():
    """Strict discrete extrema only; plateaus and the end points are not extrema."""
    h = [3.0, 2.0, 1.0, 2.0, 3.0, 2.0, 2.0, 1.0, 1.5]
    assert PCFOracle.extrema(h) == [2, 4, 7]
    assert PCFOracle.extrema([1.0, 2.0]) == []


# ------------------------------------------------------------------ DMD schedule (§6.2)
def _affine_system(n=60, mu=0.97, seed=3):
    """psi_{t+1} = psi* + mu (psi_t - psi*), cost ||psi - psi*||: J_t = J_0 mu^t exactly, and
    DMD of any window recovers psi* (one decaying mode plus the steady one)."""
    rng = np.random.default_rng(seed)
    star = rng.standard_normal(n)
    d0 = rng.standard_normal(n)
    cost = lambda p: float(np.linalg.norm(p - star))

    def step(u, k):
        hist = []
        for _ in range(k):
            hist.append(cost(u))
            u = star + mu * (u - star)
        return u, hist
    return star + d0, star, step, cost, mu


def test_dmd_schedule_jump_times_closed_form():
    """J_t = J_0 mu^t: the first jump is at the first chunk end t = c spacing with a full window
    (c >= snapshots) and J_{t-1} < j_start; it lands on psi*, so the run converges right
    after it.  With a threshold never met there is no jump."""
    u0, star, step, cost, mu = _affine_system()
    J0 = cost(u0)
    snapshots, spacing, j_start = 5, 7, 0.3 * J0
    ident = lambda p: p
    u, conv, J, jumps = dmd.run_schedule(u0, step, ident, ident, cost, 400, 1e-9, snapshots, spacing, 50,
                                         j_start, 1e-12)
    c = snapshots
    while J0 * mu ** (c * spacing - 1) >= j_start:
        c += 1
    assert jumps == [c * spacing]
    assert conv == c * spacing and J < 1e-9
    u, conv, J, jumps = dmd.run_schedule(u0, step, ident, ident, cost, 300, 1e-30, snapshots, spacing, 50,
                                         1e-30, 1e-12)
    assert jumps == [] and conv == -1 and abs(J - J0 * mu ** 299) < 1e-12 * J0


def test_dmd_schedule_gap_and_fixed_period():
    """A cost that never converges (tol below rounding): jumps every snapshots * spacing steps
    with no threshold and no gap (the fixed-period schedule), and every
    gap + snapshots * spacing steps after the first with a gap (rounded up to whole chunks)."""
    u0, star, step, cost, mu = _affine_system()
    ident = lambda p: p
    jitter = lambda p: p + 1e-3   # keeps the jump off psi*, so the descent goes on
    _, _, _, jumps = dmd.run_schedule(u0, step, ident, jitter, cost, 200, 1e-300, 4, 10, 0, np.inf, 1e-12)
    assert jumps == [40, 80, 120, 160, 200]
    _, _, _, jumps = dmd.run_schedule(u0, step, ident, jitter, cost, 300, 1e-300, 4, 10, 25, np.inf, 1e-12)
    assert jumps == [40, 40 + 30 + 40, 40 + 2 * 70, 40 + 3 * 70]


# ------------------------------------------------------------------ the norm of J
def _mode_field(o, comp, m, p, g):
    """Coefficients of the real field cos(2 pi (m x/Lx + p z/Lz)) g(y) e_comp (g: Chebyshev
    coefficients), written directly in the storage layout: the p = 0 plane holds the two
    halves at +-m, a p > 0 mode holds half (its conjugate at -p is implied)."""
    a = np.zeros((3, o.Mx, o.Mz, o.N + 1), np.complex128)
    gc = np.zeros(o.N + 1)
    gc[: len(g)] = g
    if m == 0 and p == 0:
        a[comp, 0, 0] = gc
    elif p == 0:
        a[comp, m % o.Mx, 0] += 0.5 * gc
        a[comp, (-m) % o.Mx, 0] += 0.5 * gc
    else:
        a[comp, m % o.Mx, p] = 0.5 * gc
    return a


# (1 - y^2) = T0/2 - T2/2; (1 - y^2)^2 = 3/8 T0 - T2/2 + T4/8; T2 itself
_ONE_MINUS_Y2 = [0.5, 0.0, -0.5]
_ONE_MINUS_Y2_SQ = [0.375, 0.0, -0.5, 0.0, 0.125]
_T2 = [0.0, 0.0, 1.0]

# Squared norms (1/(2 Lx Lz)) int |u|^2 in closed form: the mean over x, z of cos^2 is 1/2
# for a non-zero wavenumber and 1 for the mean mode; int (1-y^2)^2 = 16/15,
# int (1-y^2)^4 = 256/315, int T2^2 = 14/15.
_NORM_CASES = [
    ((0, 0, 0, _ONE_MINUS_Y2), 0.5 * 16.0 / 15.0),          # mean streamwise profile: 8/15
    ((0, 1, 0, _ONE_MINUS_Y2), 0.5 * 0.5 * 16.0 / 15.0),    # one x-mode: 4/15
    ((2, 0, 1, _ONE_MINUS_Y2), 0.5 * 0.5 * 16.0 / 15.0),    # one z-mode (p > 0, Hermitian half): 4/15
    ((1, -1, 2, _ONE_MINUS_Y2_SQ), 0.5 * 0.5 * 256.0 / 315.0),  # oblique mode: 64/315
    ((2, 0, 0, _T2), 0.5 * 14.0 / 15.0),                    # pure Chebyshev mean field: 7/15
]


def _norm_closed_form_gap(o):
    """Largest relative error of o.norm()^2 against the closed forms, one case at a time
    and for their sum (distinct modes or components are orthogonal, so squares add)."""
    gaps = []
    total, want_total = 0, 0.0
    for (comp, m, p, g), want in _NORM_CASES:
        a = _mode_field(o, comp, m, p, g)
        gaps.append(abs(o.norm(a) ** 2 - want) / want)
        total = total + a
        want_total += want
    gaps.append(abs(o.norm(total) ** 2 - want_total) / want_total)
    return max(gaps)


@pytest.mark.parametrize("grid", [(16, 17, 16), (32, 33, 48), (48, 25, 32)])
def test_norm_closed_forms(grid):
    """||u||^2 = (1/(2 Lx Lz)) int |u|^2 (the norm of J = ||r1||): exact values of single
    mean, x, z and oblique modes and of a pure Chebyshev profile."""
    assert _norm_closed_form_gap(PCFOracle(*grid)) < 1e-14


class _NormWithoutHalf(PCFOracle):
    def norm_phys(self, val):
        return math.sqrt(2.0) * PCFOracle.norm_phys(self, val)


class _NormSumOverXZ(PCFOracle):
    def norm_phys(self, val):
        s = (val ** 2).sum(axis=0).sum(axis=(-2, -1))
        return math.sqrt(0.5 * float((self.w_cc * s).sum()))


class _NormUniformInY(PCFOracle):
    def norm_phys(self, val):
        s = (val ** 2).sum(axis=0).mean(axis=(-2, -1))
        return math.sqrt(0.5 * float(s.sum() * 2.0 / len(s)))


@pytest.mark.parametrize("bad", [_NormWithoutHalf, _NormSumOverXZ, _NormUniformInY])
def test_norm_closed_forms_catch_planted_mistakes(bad):
    """A dropped 1/2, a sum in place of the mean over x, z, or uniform weights in y miss the
    closed forms by far more than rounding."""
    assert _norm_closed_form_gap(bad(16, 17, 16)) > 1e-2


# ------------------------------------------------------------------ equilibria: shifts, alignment, dissipation
from oracle import equilibria as eqm  # noqa: E402


def test_shift_by_grid_points_is_a_roll(o16):
    """A shift by whole grid spacings moves the physical values by whole points."""
    a = gi.random_perturbation(16, 17, 16, 0.1, 5)
    for i, j in [(1, 0), (0, 3), (5, 7), (15, 15)]:
        b = eqm.shift(o16, a, i * LX / 16, j * LZ / 16)
        want = np.roll(o16.to_phys(a), (i, j), axis=(-2, -1))
        assert np.max(np.abs(o16.to_phys(b) - want)) < 1e-14


def test_shift_of_a_single_mode(o16):
    """Any shift of one (m, p, n) mode equals the closed form 2 Re(c T_n e^{i(kx (x - lx) + kz (z - lz))})."""
    x = np.arange(16) * LX / 16
    z = np.arange(16) * LZ / 16
    a = np.zeros((3, o16.Mx, o16.Mz, o16.N + 1), np.complex128)
    c = 0.3 - 0.7j
    a[1, 2, 3, 4] = c
    lx, lz = 0.37 * LX, 0.81 * LZ
    got = o16.to_phys(eqm.shift(o16, a, lx, lz))[1]
    E = np.exp(1j * (o16.kx[2] * (x[:, None] - lx) + o16.kz[3] * (z[None, :] - lz)))
    want = 2 * np.real(c * E)[None] * np.cos(4 * np.arccos(o16.y))[:, None, None]
    assert np.max(np.abs(got - want)) < 1e-14


@pytest.mark.parametrize("seed", [0, 1])
def test_align_recovers_a_shift(o16, seed):
    """A field and a shifted copy: alignment finds the inverse shift and distance zero."""
    rng = np.random.default_rng(seed)
    a = gi.random_perturbation(16, 17, 16, 0.1, 10 + seed)
    lx0, lz0 = rng.uniform(0, LX), rng.uniform(0, LZ)
    b = eqm.shift(o16, a, lx0, lz0)
    lx, lz, bs, dist = eqm.align(o16, a, b)
    assert dist < 1e-12
    assert abs(((lx + lx0 + LX / 2) % LX) - LX / 2) < 1e-8
    assert abs(((lz + lz0 + LZ / 2) % LZ) - LZ / 2) < 1e-8


def test_dissipation_closed_forms(o16):
    """D/D_lam = 1 for the laminar flow, 7/3 for u = (1 - y^2) e_x, and
    1 + (kx^2 16/15 + 8/3)/4 for u = cos(kx x)(1 - y^2) e_x."""
    zero = np.zeros((3, o16.Mx, o16.Mz, o16.N + 1), np.complex128)
    assert abs(eqm.dissipation(o16, zero) - 1.0) < 1e-15
    a = _mode_field(o16, 0, 0, 0, _ONE_MINUS_Y2)
    assert abs(eqm.dissipation(o16, a) - 7.0 / 3.0) < 1e-14
    b = _mode_field(o16, 0, 1, 0, _ONE_MINUS_Y2)
    kx = o16.kx[1]
    assert abs(eqm.dissipation(o16, b) - (1.0 + 0.25 * (kx * kx * 16.0 / 15.0 + 8.0 / 3.0))) < 1e-14
