"""The C-ABI library builds, loads and exports every entry point include/pcfadj.h declares
(no compute call: this runs without a GPU)."""
import ctypes
import os
import re

import pytest
from tests.paper_values import paper_values

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "pcfadj.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(pcf_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    import torch  # noqa: F401
    from paper_2306_00165_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_paper_operations():
    names = _declared()
    for op in ("pcf_residual", "pcf_adjoint_gradient", "pcf_influence_matrix_solve", "pcf_descent_step",
               "pcf_dmd_extrapolate"):
        assert op in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_host_only_queries(lib):
    lib.pcf_state_len.restype = ctypes.c_longlong
    lib.pcf_psi_len.restype = ctypes.c_longlong
    lib.pcf_status_str.restype = ctypes.c_char_p
    assert lib.pcf_abi_version() == 3
    assert lib.pcf_state_len(32, 33, 32) == 3 * 19 * 10 * 33
    assert lib.pcf_state_len(30, 33, 32) == 0          # 30 = 2*3*5 has a radix-5 factor
    assert lib.pcf_state_len(32, 32, 32) == 0          # even ny rejected
    pv = paper_values()
    assert lib.pcf_psi_len(pv["nx"], pv["ny"], pv["nz"]) == pv["snapshot_dim"]  # §6.2
    assert lib.pcf_status_str(1) == b"invalid argument"


def test_create_rejects_bad_params_without_gpu(lib):
    import paper_2306_00165_gb300 as pcf
    pcf.load_library()
    p = pcf._Params(32, 32, 32, 1, 1.0, 1.0, 400.0, 0.25, 0.25, 0, 0, 0, 0)
    h = ctypes.c_void_p()
    assert pcf._lib.pcf_create(ctypes.byref(p), None, ctypes.byref(h)) == 1   # PCF_EINVAL, before any CUDA call
    assert not h.value
    # solve_kind runs 0..5 (5: the banded sweeps with one thread per chain)
    p = pcf._Params(32, 33, 32, 1, 1.0, 1.0, 400.0, 0.25, 0.25, 0, 0, 6, 0)
    assert pcf._lib.pcf_create(ctypes.byref(p), None, ctypes.byref(h)) == 1
    assert not h.value
    # the suction boundary layer needs a finite suction length > 0, and s1 maps it to blowing
    for delta, sym in ((0.0, 0), (-0.5, 0), (float("nan"), 0), (float("inf"), 0), (0.5, pcf.SYM_S1)):
        p = pcf._Params(32, 33, 32, 1, 1.0, 1.0, 400.0, 0.25, 0.25, 0, 0, 0, pcf.ASBL, sym, 0, 0, delta)
        assert pcf._lib.pcf_create(ctypes.byref(p), None, ctypes.byref(h)) == 1
        assert not h.value
