"""FP64 reference of the learned proposal network (test infrastructure only).

A Fourier-space neural operator on the spectral coefficients of the state.  Each retained
Fourier mode mp carries F = NY*4 input values: per Chebyshev index n the channels
(Re v, Im v, Re eta, Im eta), eta = i kz u - i kx w, or (u, w, 0, 0) for the mean mode.
With X in R^{MP x S x F} (S samples) and width W:

  H0          = X[mp] E[mp]^T + bE                         (per-mode encoder, F -> W)
  Z_l[mp]     = H_{l-1}[mp] (R_l[mp] + L_l)^T + b_l        (per-mode spectral weights R_l,
  H_l         = H_{l-1} + GELU(Z_l),  l = 1..L              shared mixing L_l, residual)
  Y[mp]       = H_L[mp] D[mp]^T + bD[mp]                   (per-mode decoder, W -> F)

GELU(z) = z Phi(z) with the normal CDF Phi.  Loss = mean((Y - T)^2).  The backward pass
below is derived by hand (no autograd).  Parameters: E [MP,W,F], bE [W], D [MP,F,W],
bD [MP,F], R_l [MP,W,W], L_l [W,W], b_l [W].
"""
import math

import numpy as np


def gelu(z):
    from scipy.special import erf
    return 0.5 * z * (1.0 + erf(z / math.sqrt(2.0)))


def gelu_grad(z):
    from scipy.special import erf
    return 0.5 * (1.0 + erf(z / math.sqrt(2.0))) + z * np.exp(-0.5 * z * z) / math.sqrt(2.0 * math.pi)


def init_params(MP, NY, W=32, L=4, seed=0, cin=4):
    rng = np.random.default_rng(seed)
    F = NY * cin
    p = {"E": rng.standard_normal((MP, W, F)) / math.sqrt(F), "bE": np.zeros(W),
         "D": rng.standard_normal((MP, F, W)) * 0.1 / math.sqrt(W), "bD": np.zeros((MP, F))}
    for l in range(L):
        p[f"R{l}"] = rng.standard_normal((MP, W, W)) * (0.5 / math.sqrt(W))
        p[f"L{l}"] = rng.standard_normal((W, W)) * (0.5 / math.sqrt(W))
        p[f"b{l}"] = np.zeros(W)
    return p


def forward(p, X, L=4):
    """X: [MP, S, NY, 4] -> (Y [MP, S, NY, 4], cache)."""
    MP, S = X.shape[:2]
    Xf = X.reshape(MP, S, -1)
    H = np.einsum("msf,mwf->msw", Xf, p["E"]) + p["bE"]
    Hs, Zs = [H], []
    for l in range(L):
        Wsum = p[f"R{l}"] + p[f"L{l}"][None]
        Z = np.einsum("msw,mvw->msv", H, Wsum) + p[f"b{l}"]
        Zs.append(Z)
        H = H + gelu(Z)
        Hs.append(H)
    Y = np.einsum("msw,mfw->msf", H, p["D"]) + p["bD"][:, None, :]
    return Y.reshape(X.shape), (Xf, Hs, Zs)


def loss_and_grads(p, X, T, L=4):
    Y, (Xf, Hs, Zs) = forward(p, X, L)
    MP, S = X.shape[:2]
    Yf, Tf = Y.reshape(MP, S, -1), T.reshape(MP, S, -1)
    n = Yf.size
    loss = float(np.mean((Yf - Tf) ** 2))
    dY = 2.0 * (Yf - Tf) / n
    g = {"D": np.einsum("msf,msw->mfw", dY, Hs[-1]), "bD": dY.sum(axis=1)}
    dH = np.einsum("msf,mfw->msw", dY, p["D"])
    for l in reversed(range(L)):
        dZ = dH * gelu_grad(Zs[l])
        g[f"b{l}"] = dZ.sum(axis=(0, 1))
        g[f"R{l}"] = np.einsum("msv,msw->mvw", dZ, Hs[l])
        g[f"L{l}"] = g[f"R{l}"].sum(axis=0)
        Wsum = p[f"R{l}"] + p[f"L{l}"][None]
        dH = dH + np.einsum("msv,mvw->msw", dZ, Wsum)
    g["E"] = np.einsum("msw,msf->mwf", dH, Xf)
    g["bE"] = dH.sum(axis=(0, 1))
    return loss, g
