"""Batched form: many guesses on uneven grids advanced by the same launches (CUDA graph per
step), per-instance convergence masks, an autotuned mode tile.  Every instance is compared
with the FP64 oracle at 1e-11, as in the single-grid tests."""
import numpy as np
import pytest

import pcf_inputs as gi
from oracle import PCFOracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
TOL = 1e-11


@pytest.fixture(scope="module")
def pcf():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2306_00165_gb300 as m
    m.load_library()
    return m


def _rel(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def _flat(states):
    return torch.from_numpy(np.concatenate([s.ravel() for s in states])).cuda()


MIXED = [(16, 17, 16, 2), (32, 33, 32, 2), (48, 49, 48, 1)]
# The paper's 32 x 31 x 32 grid: N = ny - 1 = 2 mod 4, so an even number of even-class
# Chebyshev rows and an odd number of odd-class rows (the other way round from MIXED)
PAPER_GRID = [(32, 31, 32, 3)]


def _mixed_inputs(grids=MIXED):
    us, seeds = [], iter(range(100))
    for (nx, ny, nz, cnt) in grids:
        for _ in range(cnt):
            us.append(gi.random_perturbation(nx, ny, nz, 0.1, next(seeds)))
    return us


def test_mixed_batch_residual_gradient_steps(pcf):
    us = _mixed_inputs()
    s = pcf.Solver.batched(MIXED)
    assert 1 <= s.mode_tile() <= 8
    u = _flat(us)
    r, J = s.residual(u)
    f = s.adjoint_gradient(u, r)
    H = s.descent_step(u, 0.01, 5).cpu().numpy()
    for b, g in enumerate(s.grids):
        o = PCFOracle(*g[:3])
        r_ref, J_ref = o.residual(us[b])
        f_ref = o.adjoint_direction(us[b], r_ref)
        assert _rel(s.view(r, b).cpu().numpy(), r_ref) <= TOL
        assert abs(float(J[b]) - J_ref) <= TOL * J_ref
        assert _rel(s.view(f, b).cpu().numpy(), f_ref) <= TOL
        ref, Href = o.run(us[b], 0.01, 5)
        assert np.max(np.abs(H[:, b] - Href) / Href) <= TOL
        assert _rel(s.view(u, b).cpu().numpy(), ref) <= TOL


def test_results_do_not_depend_on_the_tile(pcf):
    us = _mixed_inputs()
    outs = []
    for mpc in (1, 3, 6):
        s = pcf.Solver.batched(MIXED, modes_per_block=mpc)
        u = _flat(us)
        s.descent_step(u, 0.01, 3)
        outs.append(u.cpu().numpy())
    assert np.array_equal(outs[0], outs[1]) and np.array_equal(outs[0], outs[2])


def test_mixed_batch_convergence_masks(pcf):
    us = _mixed_inputs()
    hists = [PCFOracle(*g[:3]).run(us[b], 0.01, 40)[1] for b, g in
             enumerate([g for g in MIXED for _ in range(g[3])])]
    # a tolerance strictly between two steps of every instance (no rounding-level ties)
    cand = sorted(np.sqrt(h[k] * h[k + 1]) for h in hists for k in range(20, 30))
    allh = np.concatenate(hists)
    tol = next(t for t in cand[len(cand) // 2:] if np.min(np.abs(allh - t) / t) > 1e-6)
    want = [int(np.argmax(h < tol)) if np.any(h < tol) else -1 for h in hists]
    s = pcf.Solver.batched(MIXED)
    u = _flat(us)
    steps, J, jumps = s.run(u, 0.01, 40, tol=tol, dmd_period=0)
    assert steps == want


def test_uneven_64_instance_batch(pcf):
    """24 x 32x33x32 + 24 x 48x49x48 + 16 x 64x65x64 in one context, five steps with
    convergence masks: two instances of each grid match the oracle, and instance 0 (a guess
    scaled down so that its J is far below the others') is stopped by its mask before the
    update of step 3 while every other instance keeps going."""
    grids = [(32, 33, 32, 24), (48, 49, 48, 24), (64, 65, 64, 16)]
    s = pcf.Solver.batched(grids)
    us = []
    k = 0
    for (nx, ny, nz, cnt) in grids:
        for _ in range(cnt):
            us.append(gi.streak_roll(nx, ny, nz, seed=k))
            k += 1
    us[0] = 0.03 * us[0]
    sample = [0, 1, 24, 25, 62, 63]
    oracles = {g: PCFOracle(*g) for g in {tuple(s.grids[b][:3]) for b in sample}}
    refs = {b: oracles[tuple(s.grids[b][:3])].run(us[b], 0.01, 5) for b in sample}
    h0 = refs[0][1]
    tol = float(np.sqrt(h0[2] * h0[3]))
    assert all(refs[b][1][4] > 10 * tol for b in sample[1:])
    u = _flat(us)
    steps, J, jumps = s.run(u, 0.01, 5, tol=tol, dmd_period=0)
    assert steps[0] == 3 and all(x == -1 for x in steps[1:]) and jumps == 0
    for b in sample:
        o = oracles[tuple(s.grids[b][:3])]
        ref = o.run(us[b], 0.01, 3)[0] if b == 0 else refs[b][0]
        got = s.view(u, b).cpu().numpy()
        assert _rel(got, ref) <= TOL, b
        if b:  # the last J is the one measured before the last update
            assert abs(J[b] - refs[b][1][4]) <= TOL * J[b]


@pytest.mark.parametrize("grids,tile", [(MIXED, 0), (MIXED, 3), (PAPER_GRID, 0)])
def test_kernel_organisations_give_the_same_bits(pcf, grids, tile):
    """The per-mode work of a step as one per-mode kernel (solve_kind 2), as analysis, solve
    and synthesis kernels (3), or as one fused half-step kernel over instance groups (4):
    the same operations per output, so the same bits.  The autotuner's choice (0) gives the
    same bits when it keeps a dense solve; the banded sweeps (variant 4) are another
    algorithm, held to the parity tolerance."""
    us = _mixed_inputs(grids)
    outs, hists, variants = [], [], []
    for kind, launches, variant in ((2, 6, 1), (3, 10, 2), (4, 7, 3), (0, None, None)):
        s = pcf.Solver.batched(grids, solve_kind=kind, modes_per_block=tile)
        if launches is not None:
            assert s.launches_per_step() == launches and s.solve_variant() == variant
            assert s.launches_per_call(3) == 1 + 3 * launches - (1 if kind == 3 else 0)
        variants.append(s.solve_variant())
        u = _flat(us)
        hists.append(s.descent_step(u, 0.01, 4).cpu().numpy())
        outs.append(u.cpu().numpy())
    for k in (1, 2, 3):   # 3: whatever group size, mode tile and organisation the autotuner picked
        if variants[k] == 4:
            assert _rel(outs[k], outs[0]) <= TOL
            assert np.max(np.abs(hists[k] - hists[0]) / hists[0]) <= TOL
            continue
        assert np.array_equal(outs[0], outs[k])
        assert np.array_equal(hists[0], hists[k])


def test_contexts_of_different_sizes_coexist(pcf):
    """A kernel's shared-memory limit belongs to the kernel, not to a context: creating a
    smaller context later must not break an earlier, larger one (its captured graph and a new
    capture give the same bits as before)."""
    big = pcf.Solver(48, 49, 48, batch=2)
    ub = torch.from_numpy(gi.batch(gi.streak_roll, range(2), 48, 49, 48)).cuda()
    u1 = ub.clone()
    H1 = big.descent_step(u1, 0.01, 2)
    for kind in (0, 4):
        small = pcf.Solver(16, 17, 16, batch=1, solve_kind=kind)
        us = torch.from_numpy(gi.batch(gi.streak_roll, range(1), 16, 17, 16)).cuda()
        small.descent_step(us, 0.01, 2)
        small.close()
    u2 = ub.clone()
    H2 = big.descent_step(u2, 0.01, 2)
    assert torch.equal(u1, u2) and torch.equal(H1, H2)
    u3 = ub.clone()
    big.descent_step(u3, 0.01, 1)
    big.descent_step(u3, 0.01, 1)
    assert torch.equal(u3, u1)
