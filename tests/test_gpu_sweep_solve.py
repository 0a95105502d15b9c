"""The descent step with the Stokes solve by banded tau sweeps, one thread per chain
(solve_kind 5, k_sweep), against the FP64 oracle at the plain FP64 tolerance: trajectories
on grids whose classes have even and odd lengths (N = 16, 32, 30, 48), a mixed batch of
three grids, the float-float form, the symmetric subspace (reduced launches over the modes
m >= 0), the suction boundary layer, a convergence mask that stops one instance, and the
DNS.  The step size of the dummy dynamics differs from dt in one case, so that the sweep
reads the second mode table."""
import numpy as np
import pytest

import pcf_inputs as gi
from oracle import PCFOracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
TOL = 1e-11
SWEEP = 5


def _rel(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


@pytest.fixture(scope="module")
def pcf():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2306_00165_gb300 as m
    m.load_library()
    return m


def _check_run(s, us, oracles, dtau, nsteps, u=None):
    u = torch.from_numpy(np.stack(us)).cuda() if u is None else u
    H = s.descent_step(u, dtau, nsteps).cpu().numpy()
    got = u.cpu().numpy()
    for b, (u0, o) in enumerate(zip(us, oracles)):
        ref, href = o.run(u0, dtau, nsteps)
        assert np.max(np.abs(H[:, b] - href) / href) <= TOL, b
        assert _rel(got[b], ref) <= TOL, b


@pytest.mark.parametrize("grid,batch", [((16, 17, 16), 2), ((32, 33, 32), 3), ((32, 31, 32), 2),
                                        ((48, 49, 48), 1), ((32, 17, 48), 2)])
def test_sweep_trajectory_matches_oracle(pcf, grid, batch):
    s = pcf.Solver(*grid, batch=batch, solve_kind=SWEEP)
    assert s.solve_variant() == 4
    o = PCFOracle(*grid)
    us = [gi.random_perturbation(*grid, 0.1, 40 + b) for b in range(batch)]
    _check_run(s, us, [o] * batch, 0.01, 6)


def test_sweep_with_a_second_step_size(pcf):
    grid = (16, 17, 16)
    s = pcf.Solver(*grid, batch=2, dt=0.25, dtau_hat=0.5, solve_kind=SWEEP)
    o = PCFOracle(*grid, dt=0.25, dtau_hat=0.5)
    us = [gi.streak_roll(*grid, seed=45 + b) for b in range(2)]
    _check_run(s, us, [o, o], 0.01, 6)


def test_sweep_mixed_batch(pcf):
    grids = [(16, 17, 16, 2), (32, 33, 32, 2), (48, 49, 48, 1)]
    s = pcf.Solver.batched(grids, solve_kind=SWEEP)
    us, k = [], 0
    for (nx, ny, nz, cnt) in grids:
        for _ in range(cnt):
            us.append(gi.random_perturbation(nx, ny, nz, 0.1, 50 + k))
            k += 1
    u = torch.from_numpy(np.concatenate([a.ravel() for a in us])).cuda()
    H = s.descent_step(u, 0.01, 5).cpu().numpy()
    for b, g in enumerate(s.grids):
        ref, href = PCFOracle(*g[:3]).run(us[b], 0.01, 5)
        assert np.max(np.abs(H[:, b] - href) / href) <= TOL
        assert _rel(s.view(u, b).cpu().numpy(), ref) <= TOL


def test_sweep_float_float(pcf):
    grid = (32, 33, 32)
    s = pcf.Solver(*grid, batch=2, precision=2, solve_kind=SWEEP)
    assert s.solve_variant() == 4
    o = PCFOracle(*grid)
    us = [gi.streak_roll(*grid, seed=55 + b) for b in range(2)]
    _check_run(s, us, [o, o], 0.01, 6)


@pytest.mark.parametrize("mask", [2, 3])
def test_sweep_symmetric_subspace(pcf, mask):
    """s2 enforced: the sweep runs over the modes m >= 0 only (reduced launch)."""
    grid = (32, 33, 32)
    o = PCFOracle(*grid)
    u0 = o.symmetrize(gi.random_perturbation(*grid, 0.1, 60), mask)
    s = pcf.Solver(*grid, batch=2, symmetry=mask, solve_kind=SWEEP)
    Kx, Mz = grid[0] // 3 - 1, grid[2] // 3
    assert s.symmetric_modes() == (Kx + 1) * Mz
    u = torch.from_numpy(np.stack([u0, u0])).cuda()
    H = s.descent_step(u, 0.01, 10).cpu().numpy()
    ref, hist = u0, []
    for _ in range(10):
        ref, J, _, _ = o.descent_step(ref, 0.01)
        ref = o.symmetrize(ref, mask)
        hist.append(J)
    for b in range(2):
        assert np.max(np.abs(H[:, b] - np.array(hist)) / np.array(hist)) <= TOL
        assert _rel(u.cpu().numpy()[b], ref) <= TOL


def test_sweep_suction_boundary_layer(pcf):
    grid = (32, 33, 32)
    o = PCFOracle(*grid, base_flow="asbl", suction_length=0.5)
    s = pcf.Solver(*grid, batch=1, base_flow=pcf.ASBL, suction_length=0.5, solve_kind=SWEEP)
    _check_run(s, [gi.streak_roll(*grid, seed=61)], [o], 0.01, 6)


def test_sweep_convergence_mask_stops_an_instance(pcf):
    """Instance 0 starts far below the tolerance that instance 1 never reaches: the mask stops
    it before its first update, and instance 1 follows the oracle."""
    grid = (16, 17, 16)
    o = PCFOracle(*grid)
    u_small = 1e-7 * gi.random_perturbation(*grid, 0.1, 62)
    u_big = gi.random_perturbation(*grid, 0.1, 63)
    J_small = o.residual(u_small)[1]
    tol = 10.0 * J_small
    assert o.residual(u_big)[1] > 1e3 * tol
    s = pcf.Solver(*grid, batch=2, solve_kind=SWEEP)
    u = torch.from_numpy(np.stack([u_small, u_big])).cuda()
    steps, J, _ = s.run(u, 0.01, 8, tol=tol, dmd_period=0)
    got = u.cpu().numpy()
    assert steps[0] == 0 and np.array_equal(got[0], u_small)
    ref, _ = o.run(u_big, 0.01, 8)
    assert _rel(got[1], ref) <= TOL


def test_sweep_dns_matches_the_dense_solve(pcf):
    """The DNS (the Stokes step as a time stepper) with the sweep and with the dense solve,
    both held to the oracle elsewhere, agree to the FP64 tolerance over 300 steps."""
    grid = (16, 17, 16)
    u0 = gi.batch(gi.random_perturbation, range(2), *grid, amplitude=0.2)
    out = {}
    for kind in (3, SWEEP):
        s = pcf.Solver(*grid, batch=2, dt=0.005, solve_kind=kind)
        u = torch.from_numpy(u0.copy()).cuda()
        H, _, _ = s.dns(u, 300)
        out[kind] = (u.cpu().numpy(), H.cpu().numpy())
    assert _rel(out[SWEEP][0], out[3][0]) <= TOL
    assert np.max(np.abs(out[SWEEP][1] - out[3][1]) / np.abs(out[3][1])) <= TOL
