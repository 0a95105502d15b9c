"""DMD (§6) and the convergence driver on the GPU against the FP64 oracle.

The snapshot vector and its inverse are exact re-arrangements (1e-13); the DMD steady
state agrees with the oracle's SVD-based DMD where the snapshot matrix is well
conditioned (synthetic affine dynamics: 1e-9); the convergence driver stops each
instance at exactly the oracle's step.
"""
import numpy as np
import pytest

import pcf_inputs as gi
from oracle import PCFOracle, dmd

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pcf():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2306_00165_gb300 as m
    m.load_library()
    return m


def _rel(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


@pytest.mark.parametrize("grid", [(16, 17, 16), (32, 33, 32), (48, 49, 48)])
def test_snapshot_round_trip(pcf, grid):
    o = PCFOracle(*grid)
    u = gi.batch(gi.streak_roll, [0, 1], *grid)
    s = pcf.Solver(*grid, batch=2)
    ud = torch.from_numpy(u).cuda()
    psi = s.snapshot(ud).cpu().numpy()
    assert psi.shape[1] == o.psi_dim()
    for b in range(2):
        assert _rel(psi[b], o.to_psi(u[b])) <= 1e-13
    back = s.from_snapshot(torch.from_numpy(psi).cuda()).cpu().numpy()
    for b in range(2):
        assert _rel(back[b], u[b]) <= 1e-13
        assert _rel(back[b], o.from_psi(psi[b])) <= 1e-13


def _affine_snapshots(o, M, r0, seed):
    rng = np.random.default_rng(seed)
    n = o.psi_dim()
    star = o.to_psi(gi.random_perturbation(o.nx, o.ny, o.nz, 0.05, seed))
    Q, _ = np.linalg.qr(rng.standard_normal((n, r0)))
    mu = np.linspace(0.5, 0.95, r0)
    a = 0.01 * rng.standard_normal(r0)
    return np.stack([star + Q @ (a * mu ** k) for k in range(M + 1)], axis=0), star


def test_dmd_affine_matches_oracle(pcf):
    grid = (16, 17, 16)
    o = PCFOracle(*grid)
    S, star = _affine_snapshots(o, 12, 5, 3)
    s = pcf.Solver(*grid, batch=1)
    out, r, J = s.dmd_extrapolate(torch.from_numpy(np.ascontiguousarray(S)).cuda(), rank_tol=1e-10)
    got = out.cpu().numpy()
    cost = lambda p: o.residual(o.from_psi(p))[1]
    psi_ref, r_ref, costs = dmd.dmd_extrapolate(S.T, cost, rank_tol=1e-10)
    assert r == r_ref
    assert abs(J - costs[r_ref]) <= 1e-9 * costs[r_ref]
    assert _rel(got, o.from_psi(psi_ref)) <= 1e-9
    # the full-rank candidate recovers the affine fixed point itself
    psi6, lam = dmd.dmd_steady_state(S.T, 6)
    assert abs(lam[0] - 1) < 1e-10 and _rel(psi6, star) < 1e-9


def test_dmd_on_descent_snapshots(pcf):
    """Snapshots every 5 steps of a 16x17x16 descent: GPU and oracle DMD pick the same rank
    and states that agree to the conditioning of the snapshot matrix."""
    grid = (16, 17, 16)
    o = PCFOracle(*grid)
    u = gi.random_perturbation(*grid, 0.1, 4)
    snaps = []
    for k in range(20):
        u, _ = o.run(u, 0.01, 5)
        snaps.append(o.to_psi(u))
    S = np.stack(snaps)
    s = pcf.Solver(*grid, batch=1)
    out, r, J = s.dmd_extrapolate(torch.from_numpy(S).cuda(), rank_tol=1e-8)
    cost = lambda p: o.residual(o.from_psi(p))[1]
    psi_ref, r_ref, costs = dmd.dmd_extrapolate(S.T, cost, rank_tol=1e-8)
    assert r == r_ref
    assert abs(J - costs[r_ref]) <= 1e-6 * costs[r_ref]
    assert _rel(out.cpu().numpy(), o.from_psi(psi_ref)) <= 1e-6


def test_run_stops_at_the_oracle_step(pcf):
    """Convergence masks: with tol set between two oracle steps, each instance stops at
    exactly the oracle's step, and later steps leave it unchanged."""
    grid = (16, 17, 16)
    o = PCFOracle(*grid)
    u0 = gi.batch(gi.random_perturbation, [0, 1, 2], *grid, 0.1)
    hists = [o.run(u0[b], 0.01, 60)[1] for b in range(3)]
    tol = 0.5 * (hists[1][40] + hists[1][41])
    want = [int(np.argmax(h < tol)) if np.any(h < tol) else -1 for h in hists]
    s = pcf.Solver(*grid, batch=3)
    ud = torch.from_numpy(u0).cuda()
    steps, J, jumps = s.run(ud, 0.01, 60, tol=tol, dmd_period=0)
    assert steps == want and jumps == 0
    got = ud.cpu().numpy()
    for b in range(3):
        if want[b] >= 0:
            ref, _ = o.run(u0[b], 0.01, want[b])
            assert _rel(got[b], ref) <= 1e-11


def test_run_with_dmd_period_matches_oracle(pcf):
    """One DMD period (20 snapshots every 5 steps, then the jump) against the oracle."""
    grid = (16, 17, 16)
    o = PCFOracle(*grid)
    u0 = gi.random_perturbation(*grid, 0.1, 6)
    s = pcf.Solver(*grid, batch=1)
    ud = torch.from_numpy(u0[None]).cuda()
    steps, J, jumps = s.run(ud, 0.01, 105, tol=1e-30, dmd_period=100, dmd_snapshots=20, rank_tol=1e-8)
    assert jumps == 1 and steps == [-1]
    u = u0.copy()
    snaps = []
    for k in range(20):
        u, _ = o.run(u, 0.01, 5)
        snaps.append(o.to_psi(u))
    cost = lambda p: o.residual(o.from_psi(p))[1]
    psi_ref, r_ref, costs = dmd.dmd_extrapolate(np.stack(snaps).T, cost, rank_tol=1e-8)
    u = o.from_psi(psi_ref)
    u, _ = o.run(u, 0.01, 5)
    assert _rel(ud.cpu().numpy()[0], u) <= 1e-6


def test_run_schedule_matches_oracle(pcf):
    """§6.2's schedule with a threshold and a gap: a sliding window of 6 snapshots every 5
    steps, the first jump once J falls below j_start (between the J of steps 39 and 44, so at
    step 45), 10 steps of gap, then a fresh collection and a second jump at step 85."""
    grid = (16, 17, 16)
    o = PCFOracle(*grid)
    u0 = gi.random_perturbation(*grid, 0.1, 7)
    _, h = o.run(u0, 0.01, 45)
    j_start = 0.5 * (h[39] + h[44])
    cost = lambda p: o.residual(o.from_psi(p))[1]
    ref, conv, Jref, jumps_ref = dmd.run_schedule(u0, lambda u, n: o.run(u, 0.01, n), o.to_psi, o.from_psi, cost,
                                                  100, 1e-30, 6, 5, 10, j_start, 1e-8)
    assert jumps_ref == [45, 85] and conv == -1
    s = pcf.Solver(*grid, batch=1)
    ud = torch.from_numpy(u0[None].copy()).cuda()
    steps, J, jumps = s.run_schedule(ud, 0.01, 100, tol=1e-30, snapshots=6, spacing=5, gap=10, j_start=j_start,
                                     rank_tol=1e-8)
    assert jumps == 2 and steps == [-1]
    assert _rel(ud.cpu().numpy()[0], ref) <= 1e-6
    assert abs(J[0] - Jref) <= 1e-6 * Jref


def test_run_schedule_without_dmd_and_bad_schedules(pcf):
    grid = (16, 17, 16)
    s = pcf.Solver(*grid, batch=2)
    u = torch.from_numpy(gi.batch(gi.random_perturbation, range(2), *grid)).cuda()
    u2 = u.clone()
    steps, J, jumps = s.run_schedule(u, 0.01, 30, tol=1e-30, dmd=False)
    s.descent_step(u2, 0.01, 30)
    assert jumps == 0 and torch.equal(u, u2)
    for bad in (dict(snapshots=2), dict(spacing=0), dict(gap=-1), dict(j_start=float("nan")), dict(rank_tol=0.0)):
        with pytest.raises(pcf.PCFError):
            s.run_schedule(u, 0.01, 10, **bad)
