"""The seeded input recipes produce admissible states (CPU).

Both the oracle and the CUDA path take their initial guesses from ``pcf_inputs``; the method
(§4) needs them in the space it works in: divergence-free velocity perturbations that vanish
at the walls, of real fields.  Each property is checked here with numpy's Chebyshev module,
independently of the generators' own helpers and of the oracle."""
import math

import numpy as np
import pytest
from numpy.polynomial import chebyshev as npC

import pcf_inputs as gi

GRIDS = [(16, 17, 16), (32, 31, 32), (32, 33, 32), (48, 49, 48)]
GENERATORS = {
    "random_perturbation": lambda g, s: gi.random_perturbation(*g, 0.1, s),
    "streak_roll": lambda g, s: gi.streak_roll(*g, seed=s),
}


def _wavenumbers(nx, nz):
    Kx, Kz = nx // 3 - 1, nz // 3 - 1
    m = np.array(list(range(Kx + 1)) + list(range(-Kx, 0)))
    kx = 2 * math.pi * m / gi.LX_PAPER
    kz = 2 * math.pi * np.arange(Kz + 1) / gi.LZ_PAPER
    return kx[:, None, None], kz[None, :, None], Kx


@pytest.mark.parametrize("name", sorted(GENERATORS))
@pytest.mark.parametrize("grid", GRIDS)
def test_inputs_are_admissible(name, grid):
    nx, ny, nz = grid
    u = GENERATORS[name](grid, 3)
    KX, KZ, Kx = _wavenumbers(nx, nz)
    scale = np.abs(u).max()
    # no slip: a(+1) = sum a_n, a(-1) = sum (-1)^n a_n for every component and mode
    sgn = (-1.0) ** np.arange(ny)
    assert np.abs(u.sum(axis=-1)).max() <= 1e-13 * scale
    assert np.abs((u * sgn).sum(axis=-1)).max() <= 1e-13 * scale
    # divergence i kx u + dv/dy + i kz w, every Chebyshev coefficient
    dv = np.pad(npC.chebder(u[1], axis=-1), [(0, 0), (0, 0), (0, 1)])
    div = 1j * KX * u[0] + dv + 1j * KZ * u[2]
    assert np.abs(div).max() <= 1e-14 * scale * ny
    # real fields: the p = 0 plane is conjugate-symmetric in m and the mean mode is real
    Mx = 2 * Kx + 1
    for i in range(1, Kx + 1):
        assert np.array_equal(u[:, Mx - i, 0], np.conj(u[:, i, 0]))
    assert np.all(u[:, 0, 0].imag == 0)
    assert np.all(u[1, 0, 0] == 0)          # no mean wall-normal velocity


@pytest.mark.parametrize("grid", GRIDS)
def test_random_perturbation_has_the_requested_norm(grid):
    """||u||^2 = (1/(2 Lx Lz)) int |u|^2 dV = (1/2) sum_modes w_p int_{-1}^{1} |a(y)|^2 dy with
    w_p = 1 for p = 0 and 2 for the p > 0 modes (their conjugates are not stored); the y
    integral is exact here (Chebyshev product and antiderivative)."""
    u = gi.random_perturbation(*grid, 0.07, 11)
    total = 0.0
    for c in range(3):
        for i in range(u.shape[1]):
            for j in range(u.shape[2]):
                a = u[c, i, j]
                prod = npC.chebmul(a.real, a.real) + npC.chebmul(a.imag, a.imag)
                anti = npC.chebint(prod)
                total += (1.0 if j == 0 else 2.0) * (npC.chebval(1.0, anti) - npC.chebval(-1.0, anti))
    assert math.isclose(math.sqrt(0.5 * total), 0.07, rel_tol=1e-12)


@pytest.mark.parametrize("name", sorted(GENERATORS))
def test_inputs_are_seeded(name):
    g = (16, 17, 16)
    a, b, c = GENERATORS[name](g, 5), GENERATORS[name](g, 5), GENERATORS[name](g, 6)
    assert np.array_equal(a, b) and not np.array_equal(a, c)


def test_batch_stacks_the_seeds():
    out = gi.batch(gi.random_perturbation, [1, 2], 16, 17, 16)
    assert out.shape[0] == 2
    assert np.array_equal(out[1], gi.random_perturbation(16, 17, 16, seed=2))
