"""Symmetric-subspace descent on the CUDA path (§5.1 symmetries s1, s2; §3.4: the descent is
equivariant under them).  The projection against the oracle's (which applies s1 and s2 on
the collocation grid), descent with the symmetries enforced against the oracle's projected
descent, preservation of the subspace without enforcement, per-instance masks in a batch,
the float-float form, and the kernel organisations."""
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


def _oracle_run(o, u0, mask, nsteps, dtau=0.01):
    u = o.symmetrize(u0, mask) if mask else u0
    hist = []
    for _ in range(nsteps):
        u, J, _, _ = o.descent_step(u, dtau)
        if mask:
            u = o.symmetrize(u, mask)
        hist.append(J)
    return u, np.array(hist)


@pytest.mark.parametrize("grid", [(16, 17, 16), (32, 33, 32), (48, 49, 48)])
@pytest.mark.parametrize("mask", [1, 2, 3])
def test_symmetrize_matches_oracle(pcf, grid, mask):
    o = PCFOracle(*grid)
    u0 = gi.random_perturbation(*grid, 0.1, 21)
    s = pcf.Solver(*grid, batch=1)
    u = torch.from_numpy(u0[None].copy()).cuda()
    s.symmetrize(u, mask)
    assert _rel(u.cpu().numpy()[0], o.symmetrize(u0, mask)) <= 1e-13


@pytest.mark.parametrize("grid", [(16, 17, 16), (32, 33, 32)])
@pytest.mark.parametrize("mask,solve_kind", [(3, 0), (3, 3), (2, 3), (1, 3), (3, 4)])
def test_enforced_descent_matches_oracle(pcf, grid, mask, solve_kind):
    """With s2 enforced and the split per-mode kernels (solve_kind 3), a step computes the
    modes m >= 0 only and rebuilds the modes m < 0 from the s2 relation (symmetric_modes);
    with s1 alone, or the fused kernel (4), it computes every mode.  Both match the
    oracle's projected descent."""
    o = PCFOracle(*grid)
    u0 = gi.random_perturbation(*grid, 0.1, 22)
    ref, href = _oracle_run(o, u0, mask, 20)
    s = pcf.Solver(*grid, batch=2, symmetry=mask, solve_kind=solve_kind)
    Kx, Mz, Mx = grid[0] // 3 - 1, grid[2] // 3, 2 * (grid[0] // 3 - 1) + 1
    if solve_kind == 3:
        assert s.symmetric_modes() == ((Kx + 1) * Mz if mask & 2 else Mx * Mz)
    if solve_kind == 4:
        assert s.symmetric_modes() == Mx * Mz
    u = torch.from_numpy(np.stack([u0, u0])).cuda()
    H = s.descent_step(u, 0.01, 20).cpu().numpy()
    for b in range(2):
        assert np.max(np.abs(H[:, b] - href) / href) <= TOL
        assert _rel(u.cpu().numpy()[b], ref) <= TOL


def test_descent_preserves_the_subspace_without_enforcement(pcf):
    """200 plain steps from a symmetric guess stay symmetric to rounding, and equal the
    enforced run to the parity tolerance."""
    grid = (16, 17, 16)
    o = PCFOracle(*grid)
    u0 = o.symmetrize(gi.random_perturbation(*grid, 0.1, 23), 3)
    plain = pcf.Solver(*grid, batch=1)
    enforced = pcf.Solver(*grid, batch=1, symmetry=3)
    a = torch.from_numpy(u0[None].copy()).cuda()
    b = a.clone()
    Ha = plain.descent_step(a, 0.01, 200).cpu().numpy()
    Hb = enforced.descent_step(b, 0.01, 200).cpu().numpy()
    assert Ha[-1, 0] < Ha[0, 0]
    pa = a.clone()
    plain.symmetrize(pa, 3)
    assert _rel(a.cpu().numpy(), pa.cpu().numpy()) <= 1e-12
    assert _rel(a.cpu().numpy(), b.cpu().numpy()) <= TOL
    assert np.max(np.abs(Ha - Hb) / Hb) <= TOL


def test_per_instance_masks_in_a_batch(pcf):
    """s1 + s2, none, and s2 on plane Poiseuille flow, in one batch: each instance follows its
    own (projected) oracle run."""
    grid = (16, 17, 16)
    s = pcf.Solver.batched([(*grid, 2, pcf.COUETTE, 3), (*grid, 1, pcf.COUETTE, 0), (*grid, 1, pcf.POISEUILLE, 2)])
    us = [gi.random_perturbation(*grid, 0.1, 30 + k) for k in range(4)]
    u = torch.from_numpy(np.concatenate([a.ravel() for a in us])).cuda()
    H = s.descent_step(u, 0.01, 8).cpu().numpy()
    setup = [("couette", 3), ("couette", 3), ("couette", 0), ("poiseuille", 2)]
    for b, (base, mask) in enumerate(setup):
        ref, href = _oracle_run(PCFOracle(*grid, base_flow=base), us[b], mask, 8)
        assert np.max(np.abs(H[:, b] - href) / href) <= TOL
        assert _rel(s.view(u, b).cpu().numpy(), ref) <= TOL


def test_float_float_form_with_symmetry(pcf):
    grid = (32, 33, 32)
    o = PCFOracle(*grid)
    u0 = gi.streak_roll(*grid, seed=24)
    ref, href = _oracle_run(o, u0, 3, 10)
    s = pcf.Solver(*grid, batch=1, precision=pcf.FLOAT_FLOAT, symmetry=3)
    u = torch.from_numpy(u0[None].copy()).cuda()
    H = s.descent_step(u, 0.01, 10).cpu().numpy()[:, 0]
    assert np.max(np.abs(H - href) / href) <= TOL
    assert _rel(u.cpu().numpy()[0], ref) <= TOL


def test_kernel_organisations_agree_with_symmetry(pcf):
    """The single per-mode kernel and the fused kernel compute every mode and project after
    the update: the bits agree.  The split kernels compute the modes m >= 0 and rebuild the
    modes m < 0 from the s2 relation: the same states to rounding, and the modes m < 0 are
    exactly the s2 images of the modes m > 0."""
    grid = (32, 33, 32)
    u0 = torch.from_numpy(gi.batch(gi.streak_roll, range(4), *grid)).cuda()
    outs = []
    for kind in (2, 4, 3):
        s = pcf.Solver(*grid, batch=4, solve_kind=kind, modes_per_block=2, symmetry=3)
        u = u0.clone()
        H = s.descent_step(u, 0.01, 5)
        outs.append((u.cpu(), H.cpu(), s.symmetric_modes()))
    assert torch.equal(outs[1][0], outs[0][0]) and torch.equal(outs[1][1], outs[0][1])
    u3, H3, modes3 = outs[2]
    Kx, Mz, Mx = 9, 10, 19
    assert modes3 == (Kx + 1) * Mz
    assert _rel(u3.numpy(), outs[0][0].numpy()) <= 1e-12
    assert np.max(np.abs(H3.numpy() - outs[0][1].numpy()) / outs[0][1].numpy()) <= 1e-12
    a = u3.numpy()
    sgn_m = (-1.0) ** np.arange(1, Kx + 1)
    e2 = np.array([1.0, 1.0, -1.0])
    mirror = e2[None, :, None, None, None] * sgn_m[None, None, :, None, None] * np.conj(a[:, :, 1:Kx + 1])
    assert np.array_equal(a[:, :, Mx - 1:Kx:-1], mirror)


def test_invalid_symmetry_requests(pcf):
    with pytest.raises(pcf.PCFError):
        pcf.Solver(16, 17, 16, symmetry=4)
    with pytest.raises(pcf.PCFError):
        pcf.Solver(16, 17, 16, base_flow=pcf.POISEUILLE, symmetry=pcf.SYM_S1)
    s = pcf.Solver(16, 17, 16)
    u = torch.zeros(s.shape, dtype=torch.complex128, device="cuda")
    with pytest.raises(pcf.PCFError):
        s.symmetrize(u, 5)
