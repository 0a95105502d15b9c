"""Pins of the FP64 network reference (oracle/fno.py) on the CPU: its hand-derived gradient
equals central finite differences of its loss for every parameter block, and a planted
mistake in the backward pass is caught."""
import numpy as np
import pytest

from oracle import fno


def _setup(seed=0):
    rng = np.random.default_rng(seed)
    MP, S, NY, W = 3, 2, 5, 4
    p = fno.init_params(MP, NY, W=W, L=2, seed=seed)
    for k in p:
        p[k] = p[k] + 0.1 * rng.standard_normal(p[k].shape)
    X = rng.standard_normal((MP, S, NY, 4))
    T = rng.standard_normal((MP, S, NY, 4))
    return p, X, T


@pytest.mark.parametrize("key", ["E", "bE", "D", "bD", "R0", "L0", "b0", "R1", "L1", "b1"])
def test_gradient_matches_finite_differences(key):
    p, X, T = _setup(1)
    _, g = fno.loss_and_grads(p, X, T, L=2)
    rng = np.random.default_rng(2)
    d = rng.standard_normal(p[key].shape)
    eps = 1e-5
    pp = {k: v.copy() for k, v in p.items()}
    pm = {k: v.copy() for k, v in p.items()}
    pp[key] = p[key] + eps * d
    pm[key] = p[key] - eps * d
    fd = (fno.loss_and_grads(pp, X, T, L=2)[0] - fno.loss_and_grads(pm, X, T, L=2)[0]) / (2 * eps)
    an = float((g[key] * d).sum())
    assert abs(fd - an) <= 1e-7 * max(1.0, abs(an))


def test_planted_backward_mistake_is_caught():
    p, X, T = _setup(3)
    good = fno.gelu_grad
    try:
        fno.gelu_grad = lambda z: 0.5 * (1.0 + np.tanh(z))       # wrong derivative
        _, g = fno.loss_and_grads(p, X, T, L=2)
    finally:
        fno.gelu_grad = good
    eps = 1e-5
    d = np.ones_like(p["R0"])
    pp = {k: v.copy() for k, v in p.items()}
    pm = {k: v.copy() for k, v in p.items()}
    pp["R0"] += eps * d
    pm["R0"] -= eps * d
    fd = (fno.loss_and_grads(pp, X, T, L=2)[0] - fno.loss_and_grads(pm, X, T, L=2)[0]) / (2 * eps)
    assert abs(fd - float((g["R0"] * d).sum())) > 1e-4 * abs(fd)
