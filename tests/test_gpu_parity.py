"""Parity of the CUDA path (through the C ABI) with the FP64 oracle, element by element.

Tolerance: 1e-11 relative per field per step (max-norm error over the field divided by
the field's max-norm), the plain FP64 bar; 200-step trajectories on the 16x17x16 grid are
compared step by step through the norm history and in chunks through the state.
"""
import numpy as np
import pytest

import pcf_inputs as gi
from oracle import PCFOracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-11


def _rel(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2306_00165_gb300 as pcf
    pcf.load_library()
    return pcf


def _to_dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda")


def _solver(lib, grid, batch, **kw):
    return lib.Solver(*grid, batch=batch, **kw)


GRIDS = [(16, 17, 16), (32, 33, 32), (48, 49, 48), (32, 17, 48), (32, 31, 32)]  # last: the paper's §5.1 grid


@pytest.mark.parametrize("grid", GRIDS)
def test_influence_matrix_solve(lib, grid):
    o = PCFOracle(*grid)
    rng = np.random.default_rng(3)
    shp = (3, o.Mx, o.Mz, o.N + 1)
    F = (rng.standard_normal(shp) + 1j * rng.standard_normal(shp)) * np.exp(-0.2 * np.arange(o.N + 1))
    F[:, o.Mx - 1:o.Kx:-1, 0] = np.conj(F[:, 1:o.Kx + 1, 0])
    F[:, 0, 0] = F[:, 0, 0].real
    s = _solver(lib, grid, 1)
    for step in (0.25,):
        got = s.influence_matrix_solve(_to_dev(F[None]), step).cpu().numpy()[0]
        ref = o.stokes_step(F, step)
        assert _rel(got, ref) <= TOL


@pytest.mark.parametrize("grid", GRIDS)
def test_residual_and_gradient(lib, grid):
    o = PCFOracle(*grid)
    seeds = [0, 1, 2]
    u = np.stack([gi.random_perturbation(*grid, 0.1, s) for s in seeds])
    s = _solver(lib, grid, len(seeds))
    ud = _to_dev(u)
    r, J = s.residual(ud)
    f = s.adjoint_gradient(ud, r)
    r, J, f = r.cpu().numpy(), J.cpu().numpy(), f.cpu().numpy()
    for b in range(len(seeds)):
        r_ref, J_ref = o.residual(u[b])
        f_ref = o.adjoint_direction(u[b], r_ref)
        assert _rel(r[b], r_ref) <= TOL
        assert abs(J[b] - J_ref) <= TOL * J_ref
        assert _rel(f[b], f_ref) <= TOL


def test_laminar_exact_zero(lib):
    grid = (16, 17, 16)
    s = _solver(lib, grid, 1)
    z = torch.zeros(s.shape, dtype=torch.complex128, device="cuda")
    r, J = s.residual(z)
    f = s.adjoint_gradient(z, r)
    assert float(J[0]) == 0.0 and torch.count_nonzero(r).item() == 0 and torch.count_nonzero(f).item() == 0


def test_descent_200_steps_config1(lib):
    """16x17x16, Re 400, seed 0, amplitude 0.1, dtau 0.01: 200 steps, J at every step,
    the state every 50 steps."""
    grid = (16, 17, 16)
    o = PCFOracle(*grid)
    u0 = gi.random_perturbation(*grid, 0.1, 0)
    s = _solver(lib, grid, 1)
    ud = _to_dev(u0[None])
    u = u0.copy()
    for chunk in range(4):
        H = s.descent_step(ud, 0.01, 50).cpu().numpy()[:, 0]
        u, Href = o.run(u, 0.01, 50)
        assert np.max(np.abs(H - Href) / Href) <= TOL
        assert _rel(ud.cpu().numpy()[0], u) <= TOL


def test_descent_batch_streak_roll_config2(lib):
    """The bench workload (32x33x32, 8 streak/roll guesses): 20 batched steps vs the oracle."""
    grid = (32, 33, 32)
    o = PCFOracle(*grid)
    u0 = gi.batch(gi.streak_roll, range(8), *grid)
    s = _solver(lib, grid, 8)
    ud = _to_dev(u0)
    H = s.descent_step(ud, 0.01, 10).cpu().numpy()
    got = ud.cpu().numpy()
    for b in (0, 5, 7):
        u, Href = o.run(u0[b], 0.01, 10)
        assert np.max(np.abs(H[:, b] - Href) / Href) <= TOL
        assert _rel(got[b], u) <= TOL


def test_outputs_admissible_large_grid(lib):
    """64x65x64 (largest grid of the batched workload): r1 and f divergence-free and zero
    at the walls to round-off, and equal to the oracle's element by element."""
    grid = (64, 65, 64)
    o = PCFOracle(*grid)
    u = gi.random_perturbation(*grid, 0.1, 9)
    s = _solver(lib, grid, 1)
    ud = _to_dev(u[None])
    r, J = s.residual(ud)
    f = s.adjoint_gradient(ud, r)
    for a in (r.cpu().numpy()[0], f.cpu().numpy()[0]):
        sc = np.max(np.abs(a))
        assert np.max(np.abs(o.divergence(a))) <= 1e-12 * sc * o.N ** 2
        for wv in o.wall_values(a):
            assert np.max(np.abs(wv)) <= 1e-13 * sc * o.N
    r_ref, J_ref, uf = o.residual(u, return_fields=True)
    f_ref = o.adjoint_direction(u, r_ref, uf)
    for c in range(3):
        assert _rel(r.cpu().numpy()[0, c], r_ref[c]) <= TOL
        assert _rel(f.cpu().numpy()[0, c], f_ref[c]) <= TOL
    assert abs(float(J[0]) - J_ref) <= TOL * J_ref
