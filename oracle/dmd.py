"""DMD steady-state extrapolation, plain FP64 (test infrastructure only).

Paper §6.1-6.2: snapshots psi_k along a descent trajectory, Psi = [psi_1..psi_M],
Psi' = [psi'_1..psi'_M] (the same snapshots one spacing later); thin SVD
Psi ~ U Sigma V^T truncated to rank r; A~ = U^T Psi' V Sigma^-1 (Eq. for the r x r
projection); dynamic modes phi_q = Psi' V Sigma^-1 v_q with eigenpairs (lambda_q, v_q)
of A~; omega_q = ln(lambda_q)/dtau; psi(tau) ~ sum_q b_q phi_q exp(omega_q tau)
(Eq. (DMD_linear_approximation)).  Sorted by |omega|, mode 1 is taken as steady
(omega_1 ~ 0) and psi_s = b_1 phi_1 approximates the equilibrium.  The truncation rank
r <= r* (rank of the snapshot matrix) is the one whose psi_s has the smallest cost.

Readings where the paper is silent: M+1 stored snapshots s_0..s_M give the M pairs
(Psi = s_0..s_{M-1}, Psi' = s_1..s_M); r* counts singular values above
``rank_tol * sigma_1``; the amplitudes b are the least-squares fit of the last
snapshot s_M; psi_s is the real part of b_1 phi_1; ties in cost go to the larger r.
"""
import numpy as np


def snapshot_rank(S, rank_tol):
    s = np.linalg.svd(S[:, :-1], compute_uv=False)
    return int((s > rank_tol * s[0]).sum())


def dmd_steady_state(S, r, dtau=1.0):
    """psi_s for truncation rank r; also returns eigenvalues sorted by |omega|."""
    Psi, Psi1 = S[:, :-1], S[:, 1:]
    U, s, Vt = np.linalg.svd(Psi, full_matrices=False)
    U, s, V = U[:, :r], s[:r], Vt[:r].T
    VS = V / s[None, :]
    Atil = U.T @ Psi1 @ VS
    lam, W = np.linalg.eig(Atil)
    omega = np.log(lam.astype(np.complex128)) / dtau
    order = np.argsort(np.abs(omega), kind="stable")
    Phi = Psi1 @ VS @ W
    b = np.linalg.lstsq(Phi, S[:, -1].astype(np.complex128), rcond=None)[0]
    q1 = order[0]
    psi_s = np.real(b[q1] * Phi[:, q1])
    return psi_s, lam[order]


def dmd_extrapolate(S, cost, rank_tol=1e-12, dtau=1.0):
    """Pick r in r*..1 minimising cost(psi_s(r)); returns (psi_s, r, costs by r)."""
    rstar = snapshot_rank(S, rank_tol)
    best = None
    costs = {}
    for r in range(rstar, 0, -1):
        psi_s, _ = dmd_steady_state(S, r, dtau)
        c = float(cost(psi_s))
        costs[r] = c
        if np.isfinite(c) and (best is None or c < best[1]):
            best = (psi_s, c, r)
    if best is None:
        return None, 0, costs
    return best[0], best[2], costs


def run_schedule(u, step, to_psi, from_psi, cost, max_steps, tol, snapshots, spacing, gap, j_start, rank_tol):
    """Descent with the DMD schedule of §6.2 (plain host loop).

    step(u, n) -> (u after n descent steps, costs J before each of them).  The run advances in
    chunks of ``spacing`` steps and stops at the first step whose J < tol.  Before the first
    extrapolation, the snapshots after every chunk fill a sliding window of the latest
    ``snapshots``; the first extrapolation happens at the first chunk end where the window is
    full and the chunk's last J < j_start (§6.2: J falls to the threshold first).  After a
    jump the descent runs ``gap`` steps (rounded up to whole chunks) and then collects
    ``snapshots`` fresh snapshots, one per chunk, before the next jump.  A jump is skipped when
    no candidate has a finite cost.

    Returns (u, steps to J < tol or -1, last J, jump steps)."""
    import collections
    window = collections.deque(maxlen=snapshots)
    phase, wait = "first", 0
    jumps, taken, J = [], 0, float("nan")
    gap_chunks = -(-gap // spacing)
    while taken < max_steps:
        n = min(spacing, max_steps - taken)
        u, hist = step(u, n)
        for s, v in enumerate(hist):
            J = v
            if v < tol:
                return u, taken + s, J, jumps
        taken += n
        if phase == "gap":
            wait -= 1
            if wait <= 0:
                phase = "collect"
            continue
        window.append(to_psi(u))
        ready = len(window) == snapshots and (phase == "collect" or J < j_start)
        if ready:
            psi, _, _ = dmd_extrapolate(np.stack(window, axis=1), cost, rank_tol)
            window.clear()
            if psi is not None:
                u = from_psi(psi)
                jumps.append(taken)
            phase, wait = ("gap", gap_chunks) if gap_chunks > 0 else ("collect", 0)
    return u, -1, J, jumps
