"""The exact gradient g_h of the discrete cost J_h = 1/2 ||r1||^2 (the discrete reading of
a gradient check against finite differences of J), and the paper's direction f against
it (CPU only).

* J_h of the PyTorch restatement equals 1/2 J^2 of the numpy oracle.
* <g_h, v> equals the centred finite difference of the numpy oracle's 1/2 J^2 along v to
  1e-6 relative, for admissible and for arbitrary directions v, with the Couette,
  Poiseuille and suction boundary layer base flows: the transposed discrete chain is right.
* The paper's f (§4 steps 3-4, Eq. (f_approximation)) is a descent direction of J_h:
  <g_h, f> < 0, at the paper's step sizes and at larger ones.
* A mistake planted in the differentiated residual (a dropped production term) fails the
  finite-difference check.
"""
import numpy as np
import pytest

import pcf_inputs as gi
from oracle import PCFOracle
from oracle.discrete_gradient import DiscreteCost, inner

GRID = (16, 17, 16)


def _half_J2(o, u):
    return 0.5 * o.residual(u)[1] ** 2


def _fd(o, u, v, eps):
    return (_half_J2(o, u + eps * v) - _half_J2(o, u - eps * v)) / (2 * eps)


def _arbitrary(o, seed):
    """Random coefficients with no wall or divergence condition (p = 0 plane real-field symmetric)."""
    rng = np.random.default_rng(seed)
    shp = (3, o.Mx, o.Mz, o.N + 1)
    a = (rng.standard_normal(shp) + 1j * rng.standard_normal(shp)) * np.exp(-0.3 * np.arange(o.N + 1))
    a[:, o.Mx - 1:o.Kx:-1, 0] = np.conj(a[:, 1:o.Kx + 1, 0])
    a[:, 0, 0] = a[:, 0, 0].real
    return 0.1 * a / o.norm(a)


def test_cost_matches_the_numpy_oracle():
    o = PCFOracle(*GRID)
    u = gi.random_perturbation(*GRID, 0.1, 1)
    assert abs(DiscreteCost(o).value(u) - _half_J2(o, u)) <= 1e-13 * _half_J2(o, u)


@pytest.mark.parametrize("base", ["couette", "poiseuille", "asbl"])
@pytest.mark.parametrize("kind", ["admissible", "arbitrary"])
def test_gradient_against_finite_differences(base, kind):
    o = PCFOracle(*GRID, base_flow=base, suction_length=0.5 if base == "asbl" else None)
    c = DiscreteCost(o)
    u = gi.streak_roll(*GRID, seed=2)
    g = c.gradient(u)
    for seed in (3, 4):
        v = gi.random_perturbation(*GRID, 0.1, seed) if kind == "admissible" else _arbitrary(o, seed)
        want = _fd(o, u, v, 1e-6)
        assert abs(inner(g, v) - want) <= 1e-6 * abs(want)


@pytest.mark.parametrize("dt", [0.25, 4.0, 64.0])
def test_papers_direction_descends_the_discrete_cost(dt):
    o = PCFOracle(*GRID, dt=dt, dtau_hat=dt)
    c = DiscreteCost(o)
    for seed in (0, 5):
        u = gi.streak_roll(*GRID, seed=seed)
        r1, _ = o.residual(u)
        f = o.adjoint_direction(u, r1)
        g = c.gradient(u)
        assert inner(g, f) < 0
        assert abs(inner(g, f) - _fd(o, u, f, 1e-6)) <= 1e-6 * abs(inner(g, f))


class _DroppedProduction(DiscreteCost):
    """M without the -U' v e_x production term."""

    def M_hat(self, u, g):
        out = []
        for i in range(3):
            conv = u[0] * g[i, 0] + u[1] * g[i, 1] + u[2] * g[i, 2]
            out.append(-self.U * g[i, 0] - conv)
        import torch
        return self.to_spec(torch.stack(out))


def test_finite_differences_catch_a_planted_mistake():
    o = PCFOracle(*GRID)
    u = gi.streak_roll(*GRID, seed=2)
    v = gi.random_perturbation(*GRID, 0.1, 3)
    g = _DroppedProduction(o).gradient(u)
    want = _fd(o, u, v, 1e-6)
    assert abs(inner(g, v) - want) > 1e-3 * abs(want)
