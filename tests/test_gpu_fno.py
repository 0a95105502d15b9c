"""Learned proposal on the GPU: the BF16/FP32-accumulate network against the FP64 reference
(oracle/fno.py), training, the judged proposal step, and what a trained network gains over
the descent without it.

Tolerances: operands are rounded to bf16 (8 significant bits, relative 2^-9 per operand)
before each product and accumulated in FP32; through four layers this gives errors of a
few 1e-3 relative in the outputs and gradients.  Asserted: 2e-2 (forward), 5e-2 (each
gradient block, relative in norm)."""
import numpy as np
import pytest

import pcf_inputs as gi
from oracle import fno as ofno

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pcf():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2306_00165_gb300 as m
    m.load_library()
    return m


def _net_and_data(pcf, MP=45, NY=17, S=4, seed=0):
    rng = np.random.default_rng(seed)
    net = pcf.FNO(MP, NY, width=32, layers=4, seed=seed)
    p = ofno.init_params(MP, NY, W=32, L=4, seed=seed)
    p["D"] = rng.standard_normal(p["D"].shape) / np.sqrt(32)
    p["bD"] = 0.1 * rng.standard_normal(p["bD"].shape)
    for l in range(4):
        p[f"b{l}"] = 0.1 * rng.standard_normal(32)
    net.set_params(net.pack(p))
    X = rng.standard_normal((MP, S, NY, 4))
    T = rng.standard_normal((MP, S, NY, 4))
    return net, p, X, T


def test_forward_matches_reference(pcf):
    net, p, X, T = _net_and_data(pcf)
    Yg = net.forward(torch.tensor(X, dtype=torch.float32, device="cuda")).cpu().numpy()
    Yr, _ = ofno.forward(p, X)
    assert np.linalg.norm(Yg - Yr) / np.linalg.norm(Yr) <= 2e-2


def test_gradients_match_reference(pcf):
    net, p, X, T = _net_and_data(pcf, seed=1)
    loss, g = net.loss_grad(torch.tensor(X, dtype=torch.float32, device="cuda"),
                            torch.tensor(T, dtype=torch.float32, device="cuda"))
    lr, gr = ofno.loss_and_grads(p, X, T)
    assert abs(loss - lr) <= 2e-2 * lr
    gg = net.unpack(g.cpu().numpy())
    for k in gr:
        err = np.linalg.norm(gg[k] - gr[k]) / max(np.linalg.norm(gr[k]), 1e-30)
        assert err <= 5e-2, (k, err)


def test_training_reduces_loss(pcf):
    rng = np.random.default_rng(5)
    MP, NY, S = 45, 17, 8
    net = pcf.FNO(MP, NY, seed=5)
    X = torch.tensor(rng.standard_normal((MP, S, NY, 4)), dtype=torch.float32, device="cuda")
    T = 0.3 * X - 0.1 * X.roll(1, dims=2)           # a learnable linear map of the inputs
    first = net.train_step(X, T, 3e-3)
    for _ in range(150):
        last = net.train_step(X, T, 3e-3)
    assert last < 0.25 * first


def test_proposals_are_judged(pcf):
    grid = (16, 17, 16)
    s = pcf.Solver(*grid, batch=4)
    u0 = gi.batch(gi.random_perturbation, range(4), *grid, 0.1)
    u = torch.from_numpy(u0).cuda()
    net = pcf.FNO(s.shape[2] * s.shape[3], grid[1], seed=7)
    acc, J0, J1 = net.propose(s, u, 10.0 * pcf.FNO.unit_scale(s))
    _, Jnow = s.residual(u)
    for b in range(4):
        assert bool(acc[b]) == (J1[b] < J0[b])
        if acc[b]:
            assert abs(float(Jnow[b]) - J1[b]) <= 1e-12 * J1[b]
        else:
            assert torch.equal(u[b], torch.from_numpy(u0[b]).cuda())


def _trajectory_pairs(pcf, grid, seeds, lag_steps, every, nsnap, dtau=0.01):
    s = pcf.Solver(*grid, batch=len(seeds))
    u = torch.from_numpy(gi.batch(gi.streak_roll, seeds, *grid)).cuda()
    feats = []
    for k in range(nsnap):
        feats.append(pcf.FNO.features(s, u).clone())
        s.descent_step(u, dtau, every)
    lag = lag_steps // every
    X = torch.cat([feats[k] for k in range(nsnap - lag)], dim=1)
    Y = torch.cat([feats[k + lag] - feats[k] for k in range(nsnap - lag)], dim=1)
    return X, Y


def test_trained_network_gain(pcf):
    """Train on descent trajectories (16x17x16, pairs 5 tau apart), then compare plain descent
    with descent that also takes a judged proposal every 250 steps (both branches relaxed 20
    steps before the comparison), on fresh guesses, for the same number of descent steps of
    the kept branch.  Reports the J ratio; a proposal is kept only when it lowers J."""
    grid = (16, 17, 16)
    dtau = 0.01
    X, Y = _trajectory_pairs(pcf, grid, list(range(1000, 1016)), 500, 50, 40, dtau)
    # per-coefficient scales: inverse RMS over the training states
    rms = X.pow(2).mean(dim=1).sqrt()
    scale = torch.where(rms > 1e-30, 1.0 / rms.clamp_min(1e-30), torch.zeros_like(rms)).contiguous()
    X, Y = X * scale[:, None], Y * scale[:, None]
    net = pcf.FNO(X.shape[0], grid[1], seed=11)
    n = X.shape[1]
    g = torch.Generator(device="cuda").manual_seed(0)
    first = None
    for it in range(400):
        idx = torch.randint(0, n, (16,), device="cuda", generator=g)
        loss = net.train_step(X[:, idx].contiguous(), Y[:, idx].contiguous(), 2e-3)
        first = loss if first is None else first
    assert loss < first
    u0 = gi.batch(gi.streak_roll, range(2000, 2008), *grid)
    plain = pcf.Solver(*grid, batch=8)
    learned = pcf.Solver(*grid, batch=8)
    up = torch.from_numpy(u0).cuda()
    ul = torch.from_numpy(u0).cuda()
    taken = 0
    for k in range(6):
        plain.descent_step(up, dtau, 250)
        learned.descent_step(ul, dtau, 250)
        acc, _, _ = net.propose(learned, ul, scale, relax_steps=20, dtau=dtau)
        plain.descent_step(up, dtau, 20)
        taken += sum(acc)
    Jp = plain.residual(up)[1].cpu().numpy()
    Jl = learned.residual(ul)[1].cpu().numpy()
    gain = float(np.exp(np.mean(np.log(Jp / Jl))))
    print(f"learned proposals taken {taken}/48, geometric-mean J(plain)/J(learned) = {gain:.3f}")
    assert taken > 0 and gain > 1.0
