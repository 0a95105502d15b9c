"""DNS with the Stokes step as a time stepper, and the guesses it yields (§5.2: the states at
the local extrema of ||u||(t)).  Parity of the trajectory, the norm history and the captured
guesses with the oracle, and the closed-form heat step of a mean-flow perturbation."""
import math

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
def pcf():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2306_00165_gb300 as m
    m.load_library()
    return m


def _oracle_dns(o, u0, nsteps):
    """Oracle trajectory with the states at the extrema of ||u||."""
    u, h, states = u0, [], []
    for _ in range(nsteps):
        states.append(u)
        h.append(o.norm(u))
        r1, _ = o.residual(u)
        u = u + o.dt * r1
    h = np.array(h)
    ext = o.extrema(h)
    return u, h, ext, [states[s] for s in ext]


def test_dns_trajectory_norms_and_guesses(pcf):
    """Two trajectories in one batch over 300 steps (four 64-step graphs and one of 44); each
    has one extremum of ||u|| in that window."""
    grid, dt = (16, 17, 16), 0.005
    o = PCFOracle(*grid, dt=dt)
    u0s = [gi.random_perturbation(*grid, 0.2, 1), gi.streak_roll(*grid, seed=1)]
    refs = [_oracle_dns(o, a, 300) for a in u0s]
    s = pcf.Solver(*grid, batch=2, dt=dt)
    u = torch.from_numpy(np.stack(u0s)).cuda()
    H, G, n = s.dns(u, 300, max_guesses=4)
    H, G, n = H.cpu().numpy(), G.cpu().numpy(), n.cpu().numpy()
    for b, (uT, h, ext, states) in enumerate(refs):
        assert len(ext) >= 1
        assert np.max(np.abs(H[:, b] - h) / h) <= 1e-12
        assert _rel(u.cpu().numpy()[b], uT) <= TOL
        assert int(n[b]) == len(ext)
        for k, st in enumerate(states):
            assert _rel(G[k, b], st) <= TOL
        assert np.count_nonzero(G[len(ext):, b]) == 0


def test_dns_guess_room_and_counts(pcf):
    """With no room for guesses the extrema are still counted; nothing else is written."""
    grid, dt = (16, 17, 16), 0.005
    s = pcf.Solver(*grid, batch=1, dt=dt)
    u = torch.from_numpy(gi.random_perturbation(*grid, 0.2, 1)[None].copy()).cuda()
    H, G, n = s.dns(u, 300, max_guesses=0)
    assert G is None and int(n[0]) == 1


def test_dns_of_a_mean_flow_perturbation_is_the_implicit_heat_step(pcf):
    grid, dt = (32, 33, 32), 0.05
    o = PCFOracle(*grid, dt=dt)
    u0 = np.zeros((3, o.Mx, o.Mz, o.ny), np.complex128)
    u0[0, 0, 0] = o.Cinv @ np.cos(0.5 * math.pi * o.y)
    u0[2, 0, 0] = 0.3 * u0[0, 0, 0]
    s = pcf.Solver(*grid, batch=1, dt=dt)
    u = torch.from_numpy(u0[None].copy()).cuda()
    H, _, _ = s.dns(u, 10)
    g = 1.0 / (1.0 + o.nu * dt * math.pi ** 2 / 4)
    assert np.max(np.abs(u.cpu().numpy()[0] - g ** 10 * u0)) < 1e-13
    h = H.cpu().numpy()[:, 0]
    assert np.allclose(h[1:] / h[:-1], g, rtol=0, atol=1e-13)


@pytest.mark.parametrize("precision", [1, 2])
def test_dns_in_the_reduced_precision_forms(pcf, precision):
    """Float-float keeps the plain tolerance; the mixed form its own per-field bound."""
    grid, dt = (32, 33, 32), 0.005
    o = PCFOracle(*grid, dt=dt)
    u0 = gi.streak_roll(*grid, seed=3)
    uT, h, _, _ = _oracle_dns(o, u0, 20)
    s = pcf.Solver(*grid, batch=1, dt=dt, precision=precision)
    u = torch.from_numpy(u0[None].copy()).cuda()
    H, _, _ = s.dns(u, 20)
    tol = TOL if precision == 2 else 1e-5
    assert _rel(u.cpu().numpy()[0], uT) <= tol
    assert np.max(np.abs(H.cpu().numpy()[:, 0] - h) / h) <= tol


def test_dns_keeps_the_symmetric_subspace(pcf):
    grid, dt = (16, 17, 16), 0.005
    o = PCFOracle(*grid, dt=dt)
    u0 = gi.random_perturbation(*grid, 0.2, 4)
    u = o.symmetrize(u0, 3)
    for _ in range(30):
        r1, _ = o.residual(u)
        u = o.symmetrize(u + dt * r1, 3)
    s = pcf.Solver(*grid, batch=1, dt=dt, symmetry=3)
    d = torch.from_numpy(u0[None].copy()).cuda()
    s.dns(d, 30)
    assert _rel(d.cpu().numpy()[0], u) <= TOL
