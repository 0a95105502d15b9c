"""The allocation-free Stokes solve (pcf_influence_matrix_solve_noalloc) against the
context-based one (pcf_influence_matrix_solve) and the oracle's dense LU, through the C ABI.

For callers that cannot allocate device memory; it keeps its tables in a static device
array shared by all calls, so calls in a row on different grids must each match the
context path and the oracle.  The largest accepted grid (64 x 65 x 64, the fullest layout
of the array, where the shared-memory cap lowers the modes per CTA) comes before a smaller
one, so stale tables from a larger call would show.  This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-11


def _rhs(o, seed):
    rng = np.random.default_rng(seed)
    shp = (3, o.Mx, o.Mz, o.N + 1)
    F = (rng.standard_normal(shp) + 1j * rng.standard_normal(shp)) * np.exp(-0.2 * np.arange(o.N + 1))
    F[:, o.Mx - 1:o.Kx:-1, 0] = np.conj(F[:, 1:o.Kx + 1, 0])
    F[:, 0, 0] = F[:, 0, 0].real
    return F


def _params(pcf, grid, batch=1, step=0.25, modes_per_block=0):
    return pcf._Params(*grid, batch, pcf.LX_PAPER, pcf.LZ_PAPER, 400.0, step, step, 0, modes_per_block, 0, 0)


def test_noalloc_matches_context_solve_two_calls():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2306_00165_gb300 as pcf
    from oracle import PCFOracle
    lib = pcf.load_library()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    calls = [((32, 33, 32), 0.25, 1, 0), ((64, 65, 64), 0.25, 3, 4), ((16, 17, 16), 0.1, 2, 0)]
    for call, (grid, step, seed, mpb) in enumerate(calls):
        o = PCFOracle(*grid)
        rhs = _rhs(o, seed)
        F = torch.from_numpy(rhs[None]).cuda()
        ref = pcf.Solver(*grid, batch=1, dt=step, dtau_hat=step).influence_matrix_solve(F, step)
        out = torch.full_like(F, float("nan"))
        p = _params(pcf, grid, 1, step, mpb)
        st = lib.pcf_influence_matrix_solve_noalloc(ctypes.byref(p), ctypes.c_void_p(F.data_ptr()),
                                                    ctypes.c_void_p(out.data_ptr()), step, stream)
        assert st == 0, f"call {call}: status {st}"
        torch.cuda.synchronize()
        a, b = out.cpu().numpy()[0], ref.cpu().numpy()[0]
        assert np.max(np.abs(a - b)) <= TOL * np.max(np.abs(b)), f"call {call}: against the context solve"
        want = o.stokes_step(rhs, step)
        assert np.max(np.abs(a - want)) <= TOL * np.max(np.abs(want)), f"call {call}: against the oracle"


def test_noalloc_rejects_oversized_requests():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2306_00165_gb300 as pcf
    lib = pcf.load_library()
    x = torch.zeros(8, dtype=torch.complex128, device="cuda")
    ptr = ctypes.c_void_p(x.data_ptr())
    for grid, batch in [((128, 97, 128), 1), ((96, 65, 96), 1), ((32, 33, 32), 2), ((64, 67, 64), 1),
                        ((128, 33, 16), 1), ((16, 33, 96), 1)]:
        p = _params(pcf, grid, batch)
        assert lib.pcf_influence_matrix_solve_noalloc(ctypes.byref(p), ptr, ptr, 0.25, None) == 1  # PCF_EINVAL
