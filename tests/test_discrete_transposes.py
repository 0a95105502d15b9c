"""Each discrete linear stage of the residual map against its explicit transpose.

The exact gradient g_h = (d r1/du)^T W r1 of the discrete cost (oracle/discrete_gradient.py)
applies the transposes of the stages of §4 steps 1-2 by reverse-mode differentiation.  Here
every linear stage on its own (the inverse x-z FFT with its 2/3 truncation, the forward FFT
and truncation, the Chebyshev collocation synthesis and analysis, the y-derivative, the
x and z derivatives, and the Stokes solve of the influence-matrix algorithm) is turned into
its explicit real matrix A by applying it to unit vectors, and its reverse-mode product
w -> A^T w is compared with the matrix transpose, together with the dot-product identity
<A v, w> = <v, A^T w> on random vectors.  A complex array enters as its real and imaginary
parts.  Grid 8x9x8 (3 x 2 retained modes, N = 8), small enough for explicit matrices.
"""
import numpy as np
import pytest
import torch

from oracle import PCFOracle
from oracle.discrete_gradient import DiscreteCost

GRID = (8, 9, 8)
TOL = 1e-12


@pytest.fixture(scope="module")
def cost():
    return DiscreteCost(PCFOracle(*GRID))


def _as_real(z):
    return torch.view_as_real(z).reshape(-1) if torch.is_complex(z) else z.reshape(-1)


def _real_map(f, shape, cplx):
    """x (real vector) -> f(x in the given shape; complex from (re, im) pairs) as a real vector."""
    def g(x):
        a = torch.view_as_complex(x.reshape(shape + (2,))) if cplx else x.reshape(shape)
        return _as_real(f(a))
    return g


def _check_stage(g, n, rng):
    eye = torch.eye(n, dtype=torch.float64)
    A = torch.stack([g(eye[k]) for k in range(n)], dim=1)  # explicit matrix, columns = images
    m = A.shape[0]
    for _ in range(2):
        v = torch.tensor(rng.standard_normal(n))
        w = torch.tensor(rng.standard_normal(m))
        x = v.clone().requires_grad_(True)
        (At_w,) = torch.autograd.grad(g(x), x, grad_outputs=w)
        ref = A.T @ w
        assert float(torch.max(torch.abs(At_w - ref))) <= TOL * float(torch.max(torch.abs(ref)))
        lhs, rhs = float(torch.dot(A @ v, w)), float(torch.dot(v, At_w))
        assert abs(lhs - rhs) <= TOL * (abs(lhs) + float(torch.linalg.norm(A @ v) * torch.linalg.norm(w)))
    return A


def _spec_shape(o):
    return (3, o.Mx, o.Mz, o.N + 1)


def test_inverse_fft_and_synthesis(cost):
    """to_phys: retained coefficients -> values on the collocation grid (Chebyshev synthesis
    in y, inverse FFTs in x and z)."""
    o = cost.o
    g = _real_map(cost.to_phys, _spec_shape(o), True)
    _check_stage(g, 2 * int(np.prod(_spec_shape(o))), np.random.default_rng(1))


def test_forward_fft_truncation_and_analysis(cost):
    """to_spec: values -> retained coefficients (forward FFTs, 2/3 truncation, Chebyshev
    analysis)."""
    o = cost.o
    shape = (3, o.ny, o.nx, o.nz)
    g = _real_map(cost.to_spec, shape, False)
    _check_stage(g, int(np.prod(shape)), np.random.default_rng(2))


@pytest.mark.parametrize("axis", ["x", "y", "z"])
def test_derivatives(cost, axis):
    """The spectral derivatives of the gradient fields: i kx, the Chebyshev derivative
    matrix, i kz."""
    o = cost.o
    D = cost.D.T.to(torch.complex128)
    f = {"x": lambda a: 1j * cost.KX * a, "y": lambda a: a @ D, "z": lambda a: 1j * cost.KZ * a}[axis]
    g = _real_map(f, _spec_shape(o), True)
    _check_stage(g, 2 * int(np.prod(_spec_shape(o))), np.random.default_rng(3))


@pytest.mark.parametrize("step", [0.25, 4.0])
def test_stokes_solve(cost, step):
    """The Stokes step S (dense tau systems per mode, influence-matrix target): rhs -> w."""
    o = cost.o
    g = _real_map(lambda F: cost.stokes_step(F, step), _spec_shape(o), True)
    _check_stage(g, 2 * int(np.prod(_spec_shape(o))), np.random.default_rng(4))
