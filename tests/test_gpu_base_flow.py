"""Plane Poiseuille base flow u_b = (1 - y^2, 0, 0) on the CUDA path (§3.1 derives the method
for a general base flow; §7 names plane Poiseuille flow).  Parity with the FP64 oracle at the
plain tolerance, a batch that mixes Couette and Poiseuille instances on one grid, the y-mirror
symmetry that the even profile implies, and the mixed-precision form at its own bound."""
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


@pytest.mark.parametrize("grid", [(16, 17, 16), (32, 33, 32)])
def test_poiseuille_residual_and_gradient(pcf, grid):
    o = PCFOracle(*grid, base_flow="poiseuille")
    u0 = gi.random_perturbation(*grid, 0.1, 8)
    s = pcf.Solver(*grid, batch=1, base_flow=pcf.POISEUILLE)
    u = torch.from_numpy(u0[None].copy()).cuda()
    r, J = s.residual(u)
    f = s.adjoint_gradient(u, r)
    r_ref, J_ref = o.residual(u0)
    f_ref = o.adjoint_direction(u0, r_ref)
    assert _rel(r.cpu().numpy()[0], r_ref) <= TOL
    assert abs(float(J[0]) - J_ref) <= TOL * J_ref
    assert _rel(f.cpu().numpy()[0], f_ref) <= TOL


def test_poiseuille_descent_trajectory(pcf):
    grid = (32, 33, 32)
    o = PCFOracle(*grid, base_flow="poiseuille")
    u0 = gi.streak_roll(*grid, seed=9)
    ref, href = o.run(u0, 0.01, 20)
    s = pcf.Solver(*grid, batch=1, base_flow=pcf.POISEUILLE)
    u = torch.from_numpy(u0[None].copy()).cuda()
    H = s.descent_step(u, 0.01, 20).cpu().numpy()[:, 0]
    assert np.max(np.abs(H - href) / href) <= TOL
    assert _rel(u.cpu().numpy()[0], ref) <= TOL


def test_poiseuille_laminar_exact_zero(pcf):
    s = pcf.Solver(16, 17, 16, batch=1, base_flow=pcf.POISEUILLE)
    u = torch.zeros(s.shape, dtype=torch.complex128, device="cuda")
    r, J = s.residual(u)
    assert float(J[0]) == 0.0 and torch.count_nonzero(r) == 0
    s.descent_step(u, 0.01, 3)
    assert torch.count_nonzero(u) == 0


def test_couette_and_poiseuille_in_one_batch(pcf):
    """Same grid, different base flows: each instance follows its own oracle."""
    grid = (16, 17, 16)
    s = pcf.Solver.batched([(*grid, 2, pcf.COUETTE), (*grid, 2, pcf.POISEUILLE)])
    us = [gi.random_perturbation(*grid, 0.1, k) for k in range(4)]
    u = torch.from_numpy(np.concatenate([a.ravel() for a in us])).cuda()
    H = s.descent_step(u, 0.01, 6).cpu().numpy()
    for b in range(4):
        o = PCFOracle(*grid, base_flow="couette" if b < 2 else "poiseuille")
        ref, href = o.run(us[b], 0.01, 6)
        assert np.max(np.abs(H[:, b] - href) / href) <= TOL
        assert _rel(s.view(u, b).cpu().numpy(), ref) <= TOL


def _mirror_y(a, N):
    sgn = (-1.0) ** np.arange(N + 1)
    out = a * sgn
    out[..., 1, :, :, :] = -out[..., 1, :, :, :]
    return out


def test_poiseuille_mirror_symmetry(pcf):
    """[u,v,w](x,y,z) -> [u,-v,w](x,-y,z) commutes with the Poiseuille descent on the GPU."""
    grid = (32, 33, 32)
    u0 = gi.random_perturbation(*grid, 0.1, 10)[None]
    s = pcf.Solver(*grid, batch=2, base_flow=pcf.POISEUILLE)
    u = torch.from_numpy(np.concatenate([u0, _mirror_y(u0, 32)])).cuda()
    s.descent_step(u, 0.01, 10, hist=False)
    a = u.cpu().numpy()
    assert _rel(_mirror_y(a[:1], 32)[0], a[1]) <= 1e-12


def test_poiseuille_mixed_precision(pcf):
    grid = (32, 33, 32)
    o = PCFOracle(*grid, base_flow="poiseuille")
    u0 = gi.random_perturbation(*grid, 0.1, 11)
    s = pcf.Solver(*grid, batch=1, precision=1, base_flow=pcf.POISEUILLE)
    u = torch.from_numpy(u0[None].copy()).cuda()
    r, J = s.residual(u)
    r_ref, J_ref = o.residual(u0)
    for c in range(3):
        assert _rel(r.cpu().numpy()[0, c], r_ref[c]) <= 1e-4
    assert abs(float(J[0]) - J_ref) <= 1e-5 * J_ref
