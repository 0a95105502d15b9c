"""Plane Poiseuille flow u_b = (1 - y^2, 0, 0) and the asymptotic suction boundary layer
u_b = (1 - exp(-(1+y)/delta), -nu/delta, 0) on the CUDA path (§3.1 derives the method for a
general base flow; §7 names both flows).  Parity with the FP64 oracle at the plain tolerance
(FP64 and float-float forms), descent trajectories, DNS, a batch that mixes all base flows
(two suction lengths) on one grid, the y-mirror symmetry of the even Poiseuille profile, s2
enforced with suction, and the mixed-precision form at its own bound."""
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


# ------------------------------------------------------------------ suction boundary layer
DELTA = 0.5   # suction length (half-heights): V = -nu/delta = -0.005 at Re 400


def _asbl(pcf, grid, batch=1, **kw):
    return pcf.Solver(*grid, batch=batch, base_flow=pcf.ASBL, suction_length=DELTA, **kw)


@pytest.mark.parametrize("grid", [(16, 17, 16), (32, 33, 32)])
@pytest.mark.parametrize("precision", [0, 2])
def test_asbl_residual_and_gradient(pcf, grid, precision):
    o = PCFOracle(*grid, base_flow="asbl", suction_length=DELTA)
    u0 = gi.random_perturbation(*grid, 0.1, 30)
    s = _asbl(pcf, grid, precision=precision)
    u = torch.from_numpy(u0[None].copy()).cuda()
    r, J = s.residual(u)
    f = s.adjoint_gradient(u, r)
    r_ref, J_ref = o.residual(u0)
    f_ref = o.adjoint_direction(u0, r_ref)
    assert _rel(r.cpu().numpy()[0], r_ref) <= TOL
    assert abs(float(J[0]) - J_ref) <= TOL * J_ref
    assert _rel(f.cpu().numpy()[0], f_ref) <= TOL


def test_asbl_descent_trajectory(pcf):
    grid = (32, 33, 32)
    o = PCFOracle(*grid, base_flow="asbl", suction_length=DELTA)
    u0 = gi.streak_roll(*grid, seed=31)
    ref, href = o.run(u0, 0.01, 20)
    s = _asbl(pcf, grid)
    u = torch.from_numpy(u0[None].copy()).cuda()
    H = s.descent_step(u, 0.01, 20).cpu().numpy()[:, 0]
    assert np.max(np.abs(H - href) / href) <= TOL
    assert _rel(u.cpu().numpy()[0], ref) <= TOL


def test_asbl_laminar_exact_zero(pcf):
    s = _asbl(pcf, (16, 17, 16))
    u = torch.zeros(s.shape, dtype=torch.complex128, device="cuda")
    r, J = s.residual(u)
    assert float(J[0]) == 0.0 and torch.count_nonzero(r) == 0
    s.descent_step(u, 0.01, 3)
    assert torch.count_nonzero(u) == 0


def test_asbl_dns(pcf):
    """The Stokes step as a DNS time stepper with the suction base flow: ||u|| history and
    final state against the oracle's DNS over 20 steps."""
    grid = (16, 17, 16)
    o = PCFOracle(*grid, base_flow="asbl", suction_length=DELTA)
    u0 = gi.random_perturbation(*grid, 0.1, 32)
    ref, href = o.dns(u0, 20)
    s = _asbl(pcf, grid)
    u = torch.from_numpy(u0[None].copy()).cuda()
    H, _, _ = s.dns(u, 20)
    assert np.max(np.abs(H.cpu().numpy()[:, 0] - href) / href) <= TOL
    assert _rel(u.cpu().numpy()[0], ref) <= TOL


def test_all_base_flows_in_one_batch(pcf):
    """Couette, Poiseuille and two suction lengths on one grid in one context: each instance
    follows its own oracle (the suction lengths get their own tables)."""
    grid = (16, 17, 16)
    kinds = [(pcf.COUETTE, "couette", None), (pcf.POISEUILLE, "poiseuille", None),
             (pcf.ASBL, "asbl", DELTA), (pcf.ASBL, "asbl", 0.25)]
    s = pcf.Solver.batched([(*grid, 1, k, 0, d or 0.0) for k, _, d in kinds])
    us = [gi.random_perturbation(*grid, 0.1, 40 + k) for k in range(4)]
    u = torch.from_numpy(np.concatenate([a.ravel() for a in us])).cuda()
    H = s.descent_step(u, 0.01, 6).cpu().numpy()
    for b, (_, name, d) in enumerate(kinds):
        ref, href = PCFOracle(*grid, base_flow=name, suction_length=d).run(us[b], 0.01, 6)
        assert np.max(np.abs(H[:, b] - href) / href) <= TOL
        assert _rel(s.view(u, b).cpu().numpy(), ref) <= TOL


def test_asbl_with_s2_enforced(pcf):
    """s2 (x shift by Lx/2, z mirror) leaves the suction profile alone: the s2-projected
    descent follows the oracle's projected descent, and its state stays in the subspace."""
    grid = (32, 33, 32)
    o = PCFOracle(*grid, base_flow="asbl", suction_length=DELTA)
    u0 = gi.random_perturbation(*grid, 0.1, 33)
    uo = o.symmetrize(u0, 2)
    href = []
    for _ in range(8):
        uo, J, _, _ = o.descent_step(uo, 0.01)
        uo = o.symmetrize(uo, 2)
        href.append(J)
    s = _asbl(pcf, grid, symmetry=pcf.SYM_S2)
    u = torch.from_numpy(u0[None].copy()).cuda()
    H = s.descent_step(u, 0.01, 8).cpu().numpy()[:, 0]
    a = u.cpu().numpy()[0]
    assert np.max(np.abs(H - np.array(href)) / np.array(href)) <= TOL
    assert _rel(a, uo) <= TOL
    assert _rel(o.symmetrize(a, 2), a) <= 1e-13


def test_asbl_rejects_s1(pcf):
    with pytest.raises(pcf.PCFError):
        _asbl(pcf, (16, 17, 16), symmetry=pcf.SYM_S1)


@pytest.mark.parametrize("plane_kernel", [0, 1])
def test_asbl_mixed_precision(pcf, plane_kernel):
    """The FP32 plane kernels (warp-register and Stockham) with the suction term."""
    grid = (32, 33, 32)
    o = PCFOracle(*grid, base_flow="asbl", suction_length=DELTA)
    u0 = gi.random_perturbation(*grid, 0.1, 34)
    s = _asbl(pcf, grid, precision=1, plane_kernel=plane_kernel)
    assert s.plane_variant() == (1 if plane_kernel == 0 else 0)
    u = torch.from_numpy(u0[None].copy()).cuda()
    r, J = s.residual(u)
    f = s.adjoint_gradient(u, r)
    r_ref, J_ref = o.residual(u0)
    f_ref = o.adjoint_direction(u0, r_ref)
    for c in range(3):
        assert _rel(r.cpu().numpy()[0, c], r_ref[c]) <= 1e-4
        assert _rel(f.cpu().numpy()[0, c], f_ref[c]) <= 1e-4
    assert abs(float(J[0]) - J_ref) <= 1e-5 * J_ref
