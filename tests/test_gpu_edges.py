"""Edge cases of the CUDA path, through the C ABI, against the FP64 oracle: zero steps, an
instance that is converged before its first step, a laminar instance inside a batch, and
a trajectory at the paper's own §5.1 parameters (32 x 31 x 32, dt = dtau_hat = 0.25,
dtau = 0.03) compared step by step at the plain FP64 tolerance."""
import math

import numpy as np
import pytest

import pcf_inputs as gi
from oracle import PCFOracle
from tests.paper_values import paper_values

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


def test_zero_steps_leave_the_state(pcf):
    u0 = gi.batch(gi.random_perturbation, [0, 1], 16, 17, 16)
    s = pcf.Solver(16, 17, 16, batch=2)
    u = torch.from_numpy(u0).cuda()
    s.descent_step(u, 0.01, 0, hist=False)
    assert np.array_equal(u.cpu().numpy(), u0)


def test_converged_before_the_first_step(pcf):
    """tol above J: each instance stops at step 0 and keeps its state bit for bit."""
    u0 = gi.batch(gi.random_perturbation, [2, 3], 16, 17, 16)
    s = pcf.Solver(16, 17, 16, batch=2)
    u = torch.from_numpy(u0).cuda()
    steps, J, jumps = s.run(u, 0.01, 50, tol=1e3, dmd_period=0)
    assert steps == [0, 0] and jumps == 0
    assert np.array_equal(u.cpu().numpy(), u0)
    o = PCFOracle(16, 17, 16)
    for b in range(2):
        assert abs(J[b] - o.residual(u0[b])[1]) <= TOL * J[b]


def test_laminar_instance_inside_a_batch(pcf):
    """u = 0 is an equilibrium: it stays exactly zero while its neighbours descend."""
    u0 = gi.batch(gi.streak_roll, [4, 5, 6], 32, 33, 32)
    u0[1] = 0.0
    s = pcf.Solver(32, 33, 32, batch=3)
    u = torch.from_numpy(u0).cuda()
    H = s.descent_step(u, 0.01, 5).cpu().numpy()
    got = u.cpu().numpy()
    assert np.all(got[1] == 0.0) and np.all(H[:, 1] == 0.0)
    o = PCFOracle(32, 33, 32)
    for b in (0, 2):
        ref, href = o.run(u0[b], 0.01, 5)
        assert np.max(np.abs(H[:, b] - href) / href) <= TOL
        assert _rel(got[b], ref) <= TOL


def test_paper_parameters_trajectory(pcf):
    """20 descent steps at the paper's §5.1 grid and step sizes, J at every step and the
    final state against the oracle."""
    pv = paper_values()
    grid = (pv["nx"], pv["ny"], pv["nz"])
    Lx, Lz = 2 * math.pi / pv["Lx_over_2pi_inverse"], 2 * math.pi / pv["Lz_over_2pi_inverse"]
    u0 = gi.streak_roll(*grid, seed=7, Lx=Lx, Lz=Lz)
    o = PCFOracle(*grid, Lx=Lx, Lz=Lz, Re=pv["Re"], dt=pv["dt"], dtau_hat=pv["dtau_hat"])
    ref, href = o.run(u0, pv["dtau"], 20)
    s = pcf.Solver(*grid, batch=1, Lx=Lx, Lz=Lz, Re=pv["Re"], dt=pv["dt"], dtau_hat=pv["dtau_hat"])
    u = torch.from_numpy(u0[None].copy()).cuda()
    H = s.descent_step(u, pv["dtau"], 20).cpu().numpy()[:, 0]
    assert np.all(np.diff(H) < 0)
    assert np.max(np.abs(H - href) / href) <= TOL
    assert _rel(u.cpu().numpy()[0], ref) <= TOL
