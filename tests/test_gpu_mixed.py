"""Mixed-precision form: FP32 x-z transforms and products, split-BF16 tensor-core Chebyshev
transforms (FP32 accumulation), FP64 tau/influence-matrix solves, FD quotients, update and
norm reductions.  Its error against the FP64 oracle is bounded by the split-BF16 contraction
(about 16 significant bits per product, 2^-16 ~ 1.5e-5, summed over the Chebyshev
coefficients) and FP32 elsewhere; measured per field it is ~1e-5.  The bound asserted here
is 1e-4 per field for r1 and f, 1e-5 for J; FP64 refinement steps continued from a mixed
state keep tracking the oracle's plain trajectory from the same seeded guess without widening
the gap.  The oracle is only ever given seeded inputs."""
import numpy as np
import pytest

import pcf_inputs as gi
from oracle import PCFOracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
MIXED_TOL = 1e-4


@pytest.fixture(scope="module")
def pcf():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2306_00165_gb300 as m
    m.load_library()
    return m


def _rel(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


@pytest.mark.parametrize("grid,plane_kernel,contraction_kernel",
                         [((16, 17, 16), 0, 0), ((16, 17, 16), 0, 1), ((32, 33, 32), 0, 0), ((32, 33, 32), 1, 1),
                          ((48, 49, 48), 0, 0), ((64, 49, 32), 0, 0), ((64, 49, 32), 1, 1), ((96, 33, 64), 0, 0),
                          ((32, 113, 32), 0, 0)])
def test_mixed_residual_and_gradient_per_field(pcf, grid, plane_kernel, contraction_kernel):
    """Both FP32 plane-kernel variants (transforms in warp registers where nx, nz allow it;
    shared-memory Stockham passes otherwise or on request) and both tensor-core paths of the
    Chebyshev transforms (tcgen05 with a tensor-memory accumulator, or mma.sync) against the
    oracle; ny = 113 fills the 128-row MMA tile."""
    o = PCFOracle(*grid)
    u = gi.batch(gi.random_perturbation, [0, 1], *grid, 0.1)
    s = pcf.Solver(*grid, batch=2, precision=1, plane_kernel=plane_kernel, contraction_kernel=contraction_kernel)
    warp_ok = grid[0] in (32, 64, 96, 128) and grid[2] in (32, 64, 96, 128)
    assert s.plane_variant() == (1 if warp_ok and plane_kernel == 0 else 0)
    assert s.contraction_variant() == 1 - contraction_kernel
    ud = torch.from_numpy(u).cuda()
    r, J = s.residual(ud)
    f = s.adjoint_gradient(ud, r)
    for b in range(2):
        r_ref, J_ref = o.residual(u[b])
        f_ref = o.adjoint_direction(u[b], r_ref)
        for c in range(3):
            assert _rel(r.cpu().numpy()[b, c], r_ref[c]) <= MIXED_TOL
            assert _rel(f.cpu().numpy()[b, c], f_ref[c]) <= MIXED_TOL
        assert abs(float(J[b]) - J_ref) <= 1e-5 * J_ref


def test_mixed_ny_limit(pcf):
    """The mixed form serves ny <= 113 (one 128-row tensor-core tile of the padded Chebyshev
    matrix); a larger ny is refused at creation, before any launch."""
    with pytest.raises(pcf.PCFError, match="not supported"):
        pcf.Solver(16, 129, 16, batch=1, precision=1)
    with pytest.raises(pcf.PCFError, match="not supported"):
        pcf.Solver(16, 115, 16, batch=1, precision=1)


def test_mixed_descent_then_fp64_refinement(pcf):
    """30 mixed steps track the oracle to 1e-5; 10 FP64 refinement steps continued on the
    GPU keep tracking the oracle's plain trajectory from the same seeded guess, without
    widening the gap.  (The oracle is only ever given seeded inputs.)"""
    grid = (32, 33, 32)
    o = PCFOracle(*grid)
    u0 = gi.streak_roll(*grid, seed=4)
    sm = pcf.Solver(*grid, batch=1, precision=1)
    ud = torch.from_numpy(u0[None]).cuda()
    H = sm.descent_step(ud, 0.01, 30).cpu().numpy()[:, 0]
    uref, Href = o.run(u0, 0.01, 30)
    assert np.max(np.abs(H - Href) / Href) <= 1e-5
    gap_mixed = _rel(ud.cpu().numpy()[0], uref)
    assert gap_mixed <= 1e-5
    s64 = pcf.Solver(*grid, batch=1, precision=0)
    H2 = s64.descent_step(ud, 0.01, 10).cpu().numpy()[:, 0]
    u2, H2ref = o.run(uref, 0.01, 10)
    assert np.max(np.abs(H2 - H2ref) / H2ref) <= 1e-5
    gap_refined = _rel(ud.cpu().numpy()[0], u2)
    assert gap_refined <= 1.5 * gap_mixed


def test_mixed_large_grid_admissible(pcf):
    """128x97x128 (the mixed workload): outputs stay divergence-free and zero at the walls in
    FP64 (the solve is FP64), and J agrees with the FP64 path to 1e-5."""
    grid = (128, 97, 128)
    o = PCFOracle(*grid)
    u = gi.random_perturbation(*grid, 0.1, 11)
    ud = torch.from_numpy(u[None]).cuda()
    r, J = pcf.Solver(*grid, batch=1, precision=1).residual(ud)
    r64, J64 = pcf.Solver(*grid, batch=1, precision=0).residual(ud)
    a = r.cpu().numpy()[0]
    sc = np.max(np.abs(a))
    assert np.max(np.abs(o.divergence(a))) <= 1e-12 * sc * o.N ** 2
    for wv in o.wall_values(a):
        assert np.max(np.abs(wv)) <= 1e-13 * sc * o.N
    assert abs(float(J[0]) - float(J64[0])) <= 1e-5 * float(J64[0])
    assert _rel(a, r64.cpu().numpy()[0]) <= MIXED_TOL
