"""Float-float form: the x-z transforms and the products in pairs of FP32 (about 48
significant bits) on the FP32 pipe, everything else FP64.  Its errors are ~1e-14 per field,
so it is held to the plain FP64 bar: 1e-11 relative per field per step against the oracle
(per-operation roundoff 2^-48 ~ 3.6e-15, through a few FFT passes, then the same
FP64 solves and amplification as the plain path)."""
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


@pytest.mark.parametrize("grid", [(16, 17, 16), (32, 33, 32), (48, 49, 48), (32, 17, 48), (32, 31, 32)])
def test_float_float_residual_and_gradient(pcf, grid):
    o = PCFOracle(*grid)
    u0 = gi.random_perturbation(*grid, 0.1, 12)
    s = pcf.Solver(*grid, batch=1, precision=pcf.FLOAT_FLOAT)
    u = torch.from_numpy(u0[None].copy()).cuda()
    r, J = s.residual(u)
    f = s.adjoint_gradient(u, r)
    r_ref, J_ref = o.residual(u0)
    f_ref = o.adjoint_direction(u0, r_ref)
    for c in range(3):
        assert _rel(r.cpu().numpy()[0, c], r_ref[c]) <= TOL
        assert _rel(f.cpu().numpy()[0, c], f_ref[c]) <= TOL
    assert abs(float(J[0]) - J_ref) <= TOL * J_ref


def test_float_float_descent_batch(pcf):
    """50 steps of the 8-guess streak/roll workload: J at every step and the final states."""
    grid = (32, 33, 32)
    u0 = gi.batch(gi.streak_roll, range(8), *grid)
    s = pcf.Solver(*grid, batch=8, precision=pcf.FLOAT_FLOAT)
    u = torch.from_numpy(u0.copy()).cuda()
    H = s.descent_step(u, 0.01, 50).cpu().numpy()
    got = u.cpu().numpy()
    o = PCFOracle(*grid)
    for b in (0, 5):
        ref, href = o.run(u0[b], 0.01, 50)
        assert np.max(np.abs(H[:, b] - href) / href) <= TOL
        assert _rel(got[b], ref) <= TOL


def test_float_float_uneven_batch_and_poiseuille(pcf):
    """An uneven batch with a Couette and a Poiseuille instance, each against its oracle."""
    s = pcf.Solver.batched([(16, 17, 16, 1, pcf.COUETTE), (32, 33, 32, 1, pcf.POISEUILLE)],
                           precision=pcf.FLOAT_FLOAT)
    us = [gi.random_perturbation(16, 17, 16, 0.1, 13), gi.random_perturbation(32, 33, 32, 0.1, 14)]
    u = torch.from_numpy(np.concatenate([a.ravel() for a in us])).cuda()
    H = s.descent_step(u, 0.01, 6).cpu().numpy()
    for b, (g, bf) in enumerate([((16, 17, 16), "couette"), ((32, 33, 32), "poiseuille")]):
        ref, href = PCFOracle(*g, base_flow=bf).run(us[b], 0.01, 6)
        assert np.max(np.abs(H[:, b] - href) / href) <= TOL
        assert _rel(s.view(u, b).cpu().numpy(), ref) <= TOL
