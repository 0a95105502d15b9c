"""Thin Python binding of libpcfadj (the GB300 adjoint-descent solver for plane Couette flow).

Argument marshalling only: every step of the method runs in the library's CUDA kernels.
PyTorch provides device memory and the current stream.  There is no CPU fallback: if the
compiled library is missing, importing the bindings raises.

Names follow the C ABI (include/pcfadj.h): residual, adjoint_gradient,
influence_matrix_solve, descent_step, dmd_extrapolate.
"""
import ctypes
import math
import os

from . import build as _build

__all__ = ["Solver", "FNO", "load_library", "state_shape", "psi_len", "probe_fp64_peak", "PCFError"]

LX_PAPER = 2.0 * math.pi / 1.14
LZ_PAPER = 2.0 * math.pi / 2.5

_lib = None


class PCFError(RuntimeError):
    pass


class _Schedule(ctypes.Structure):
    _fields_ = [("snapshots", ctypes.c_int), ("spacing", ctypes.c_int), ("gap", ctypes.c_int),
                ("j_start", ctypes.c_double), ("rank_tol", ctypes.c_double)]


class _Params(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int), ("batch", ctypes.c_int),
                ("Lx", ctypes.c_double), ("Lz", ctypes.c_double), ("Re", ctypes.c_double),
                ("dt", ctypes.c_double), ("dtau_hat", ctypes.c_double),
                ("precision", ctypes.c_int), ("modes_per_block", ctypes.c_int),
                ("solve_kind", ctypes.c_int), ("base_flow", ctypes.c_int), ("symmetry", ctypes.c_int),
                ("plane_kernel", ctypes.c_int), ("contraction_kernel", ctypes.c_int),
                ("suction_length", ctypes.c_double)]

# laminar base flows: u_b = (y,0,0), (1-y^2,0,0), and the asymptotic suction boundary layer
# (1 - exp(-(1+y)/delta), -nu/delta, 0) with delta = suction_length
COUETTE, POISEUILLE, ASBL = 0, 1, 2
SYM_S1, SYM_S2 = 1, 2        # symmetries of §5.1 (bit mask): shift-and-rotate, shift-and-reflect
FP64, MIXED, FLOAT_FLOAT = 0, 1, 2   # precision forms (pcf_precision)


def load_library(path=None):
    """Load the in-tree libpcfadj.so (built by ``build.build()``); raises if absent."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or _build.LIB
    if not os.path.exists(path):
        raise PCFError(f"libpcfadj.so not found at {path}; run __graft_entry__.build() first")
    lib = ctypes.CDLL(path)
    P = ctypes.c_void_p
    D = ctypes.c_double
    I = ctypes.c_int
    sigs = {
        "pcf_abi_version": (I, []),
        "pcf_status_str": (ctypes.c_char_p, [I]),
        "pcf_state_len": (ctypes.c_longlong, [I, I, I]),
        "pcf_psi_len": (ctypes.c_longlong, [I, I, I]),
        "pcf_create": (I, [ctypes.POINTER(_Params), P, ctypes.POINTER(P)]),
        "pcf_destroy": (None, [P]),
        "pcf_batch_create": (I, [ctypes.POINTER(_Params), I, P, ctypes.POINTER(P)]),
        "pcf_state_offset": (ctypes.c_longlong, [P, I]),
        "pcf_mode_tile": (I, [P]),
        "pcf_residual": (I, [P, P, P, P]),
        "pcf_adjoint_gradient": (I, [P, P, P, P]),
        "pcf_influence_matrix_solve": (I, [P, P, P, D]),
        "pcf_influence_matrix_solve_noalloc": (I, [ctypes.POINTER(_Params), P, P, D, P]),
        "pcf_descent_step": (I, [P, P, D, I, P]),
        "pcf_descent_step_host": (I, [P, P, D, I, P]),
        "pcf_snapshot": (I, [P, P, P]),
        "pcf_from_snapshot": (I, [P, P, P]),
        "pcf_symmetrize": (I, [P, P, I]),
        "pcf_norm": (I, [P, P, P]),
        "pcf_dns": (I, [P, P, I, P, P, I, P]),
        "pcf_dmd_extrapolate": (I, [P, P, ctypes.c_longlong, I, D, P, ctypes.POINTER(I), ctypes.POINTER(D)]),
        "pcf_run": (I, [P, P, D, I, D, I, I, D, P, P, ctypes.POINTER(I)]),
        "pcf_run_schedule": (I, [P, P, D, I, D, ctypes.POINTER(_Schedule), P, P, ctypes.POINTER(I)]),
        "pcf_probe_fp64_peak": (I, [P, ctypes.POINTER(D)]),
        "pcf_fno_create": (I, [I, I, I, I, ctypes.c_ulonglong, P, ctypes.POINTER(P)]),
        "pcf_fno_destroy": (None, [P]),
        "pcf_fno_num_params": (ctypes.c_longlong, [P]),
        "pcf_fno_set_params": (I, [P, P]),
        "pcf_fno_get_params": (I, [P, P]),
        "pcf_fno_forward": (I, [P, P, I, P]),
        "pcf_fno_loss_grad": (I, [P, P, P, I, ctypes.POINTER(D), P]),
        "pcf_fno_train_step": (I, [P, P, P, I, ctypes.c_float, ctypes.POINTER(D)]),
        "pcf_fno_features": (I, [P, P, P, P]),
        "pcf_fno_propose": (I, [P, P, P, P, I, D, P, P, P]),
        "pcf_set_kernel_timing": (I, [P, I]),
        "pcf_kernel_times": (I, [P, P, P, I]),
        "pcf_launches_per_step": (I, [P]),
        "pcf_launches_per_call": (ctypes.c_longlong, [P, I]),
        "pcf_split_config": (I, [P, ctypes.POINTER(I)]),
        "pcf_solve_variant": (I, [P]),
        "pcf_plane_variant": (I, [P]),
        "pcf_contraction_variant": (I, [P]),
        "pcf_symmetric_modes": (I, [P]),
    }
    for name, (res, args) in sigs.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _check(st):
    if st != 0:
        raise PCFError(f"pcfadj: {_lib.pcf_status_str(st).decode()} (status {st})")


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def _stream():
    import torch
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def state_shape(nx, ny, nz, batch=1):
    Kx, Kz = nx // 3 - 1, nz // 3 - 1
    return (batch, 3, 2 * Kx + 1, Kz + 1, ny)


def psi_len(nx, ny, nz):
    return int(load_library().pcf_psi_len(nx, ny, nz))


def probe_fp64_peak():
    """Measured FP64 FMA throughput of the current GPU in GFLOP/s."""
    lib = load_library()
    g = ctypes.c_double()
    _check(lib.pcf_probe_fp64_peak(_stream(), ctypes.byref(g)))
    return g.value


class Solver:
    """One grid, ``batch`` instances; all tensors are complex128 on the current CUDA device,
    shaped [batch, 3, Mx, Mz, ny] (see include/pcfadj.h for the layout).

    ``Solver.batched([(nx, ny, nz, count), ...])`` builds a heterogeneous batch instead; its
    states are one flat complex128 tensor (``flat_len`` values, instance views via ``view``)."""

    KERNEL_CLASSES = ["ysynth", "xzsynth_u", "prod_M", "mode_phi", "xzsynth_q", "prod_N", "mode_psi",
                      "yanalysis", "ysynth_step", "jnorm", "symmetrize", "dns_aux", "cheb_synth_tc",
                      "cheb_analysis_tc"]

    def __init__(self, nx, ny, nz, batch=1, Lx=LX_PAPER, Lz=LZ_PAPER, Re=400.0, dt=0.25, dtau_hat=0.25,
                 precision=0, modes_per_block=0, solve_kind=0, base_flow=COUETTE, symmetry=0, plane_kernel=0,
                 contraction_kernel=0, suction_length=0.0):
        import torch
        self.lib = load_library()
        self.shape = state_shape(nx, ny, nz, batch)
        self.nx, self.ny, self.nz, self.batch = nx, ny, nz, batch
        self.dt, self.dtau_hat = dt, dtau_hat
        p = _Params(nx, ny, nz, batch, Lx, Lz, Re, dt, dtau_hat, precision, modes_per_block, solve_kind, base_flow,
                    symmetry, plane_kernel, contraction_kernel, suction_length)
        h = ctypes.c_void_p()
        _check(self.lib.pcf_create(ctypes.byref(p), _stream(), ctypes.byref(h)))
        self._h = h
        self.device = torch.device("cuda", torch.cuda.current_device())
        self.flat = False

    @classmethod
    def batched(cls, grids, Lx=LX_PAPER, Lz=LZ_PAPER, Re=400.0, dt=0.25, dtau_hat=0.25, modes_per_block=0,
                solve_kind=0, precision=0):
        """grids: list of (nx, ny, nz, count[, base_flow[, symmetry[, suction_length]]])."""
        import torch
        self = cls.__new__(cls)
        self.lib = load_library()
        arr = (_Params * len(grids))()
        for k, g in enumerate(grids):
            nx, ny, nz, cnt = g[:4]
            arr[k] = _Params(nx, ny, nz, cnt, Lx, Lz, Re, dt, dtau_hat, precision, modes_per_block if k == 0 else 0,
                             solve_kind, g[4] if len(g) > 4 else COUETTE, g[5] if len(g) > 5 else 0, 0, 0,
                             g[6] if len(g) > 6 else 0.0)
        h = ctypes.c_void_p()
        _check(self.lib.pcf_batch_create(arr, len(grids), _stream(), ctypes.byref(h)))
        self._h = h
        self.device = torch.device("cuda", torch.cuda.current_device())
        self.grids = [g for g in grids for _ in range(g[3])]
        self.batch = len(self.grids)
        self.offsets = [int(self.lib.pcf_state_offset(h, b)) for b in range(self.batch + 1)]
        self.flat_len = self.offsets[-1]
        self.shape = (self.flat_len,)
        self.flat = True
        self.dt, self.dtau_hat = dt, dtau_hat
        return self

    def view(self, flat, b):
        """Instance b of a flat batch tensor as [3, Mx, Mz, ny]."""
        nx, ny, nz = self.grids[b][:3]
        return flat[self.offsets[b]:self.offsets[b + 1]].view(state_shape(nx, ny, nz, 1)[1:])

    def mode_tile(self):
        return int(self.lib.pcf_mode_tile(self._h))

    def close(self):
        if getattr(self, "_h", None):
            self.lib.pcf_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _chk(self, t):
        import torch
        if t.dtype != torch.complex128 or not t.is_cuda or not t.is_contiguous() or tuple(t.shape) != self.shape:
            raise PCFError(f"expected contiguous complex128 CUDA tensor of shape {self.shape}, got "
                           f"{t.dtype} {tuple(t.shape)} on {t.device}")
        return t

    def empty(self):
        import torch
        return torch.empty(self.shape, dtype=torch.complex128, device=self.device)

    def residual(self, u, r=None, with_norm=True):
        """Steps 1-2 of §4: returns (r1, J) with J a float64 tensor of length batch."""
        import torch
        self._chk(u)
        r = self.empty() if r is None else self._chk(r)
        J = torch.empty(self.batch, dtype=torch.float64, device=self.device) if with_norm else None
        _check(self.lib.pcf_residual(self._h, _ptr(u), _ptr(r), _ptr(J)))
        return r, J

    def adjoint_gradient(self, u, r, f=None):
        """Steps 3-4 of §4: the descent direction f."""
        self._chk(u)
        self._chk(r)
        f = self.empty() if f is None else self._chk(f)
        _check(self.lib.pcf_adjoint_gradient(self._h, _ptr(u), _ptr(r), _ptr(f)))
        return f

    def influence_matrix_solve(self, rhs, step, out=None):
        """One influence-matrix Stokes step: (1/step - nu Lap) out + grad p = rhs."""
        self._chk(rhs)
        out = self.empty() if out is None else self._chk(out)
        _check(self.lib.pcf_influence_matrix_solve(self._h, _ptr(rhs), _ptr(out), float(step)))
        return out

    def descent_step(self, u, dtau, nsteps=1, hist=True):
        """nsteps descent steps in place on u; returns the J history [nsteps, batch] (or None)."""
        import torch
        self._chk(u)
        H = torch.empty((nsteps, self.batch), dtype=torch.float64, device=self.device) if hist else None
        _check(self.lib.pcf_descent_step(self._h, _ptr(u), float(dtau), int(nsteps), _ptr(H)))
        return H

    def descent_step_host(self, u_host, dtau, nsteps=1, hist_host=None):
        """Same as descent_step with host (CPU, ideally pinned) complex128 tensors; synchronises."""
        _check(self.lib.pcf_descent_step_host(self._h, _ptr(u_host), float(dtau), int(nsteps),
                                              _ptr(hist_host)))

    def snapshot(self, u, psi=None):
        """Snapshot vectors of §6.2: float64 [batch, psi_len]."""
        import torch
        self._chk(u)
        n = psi_len(self.nx, self.ny, self.nz)
        psi = torch.empty((self.batch, n), dtype=torch.float64, device=self.device) if psi is None else psi
        _check(self.lib.pcf_snapshot(self._h, _ptr(u), _ptr(psi)))
        return psi

    def from_snapshot(self, psi, u=None):
        u = self.empty() if u is None else self._chk(u)
        _check(self.lib.pcf_from_snapshot(self._h, _ptr(psi), _ptr(u)))
        return u

    def norm(self, u):
        """Volume-normalised L2 norm of every instance: float64 tensor [batch]."""
        import torch
        self._chk(u)
        out = torch.empty(self.batch, dtype=torch.float64, device=self.device)
        _check(self.lib.pcf_norm(self._h, _ptr(u), _ptr(out)))
        return out

    def symmetrize(self, u, mask):
        """Project u in place onto the subspace invariant under the symmetries of mask (§5.1)."""
        self._chk(u)
        _check(self.lib.pcf_symmetrize(self._h, _ptr(u), int(mask)))
        return u

    def dns(self, u, nsteps, max_guesses=0, hist=True):
        """nsteps of u <- u^dt (the Stokes step as a DNS time stepper), in place on u.
        Returns (||u|| history [nsteps, batch], guesses [max_guesses, *state shape] or None,
        extrema found per instance as an int32 tensor [batch])."""
        import torch
        self._chk(u)
        H = torch.empty((nsteps, self.batch), dtype=torch.float64, device=self.device) if hist else None
        G = (torch.zeros((max_guesses,) + tuple(self.shape), dtype=torch.complex128, device=self.device)
             if max_guesses > 0 else None)
        n = torch.zeros(self.batch, dtype=torch.int32, device=self.device)
        _check(self.lib.pcf_dns(self._h, _ptr(u), int(nsteps), _ptr(H), _ptr(G), int(max_guesses), _ptr(n)))
        return H, G, n

    def dmd_extrapolate(self, snapshots, rank_tol=1e-12, out=None, ld=None):
        """DMD steady state of §6 from snapshots (float64 [M+1, psi_len] rows = snapshots, or a
        strided view with column stride ``ld``); returns (state [1, ...] view of ``out``, rank, J)."""
        import torch
        n = psi_len(self.nx, self.ny, self.nz)
        M = snapshots.shape[0] - 1
        ld = n if ld is None else ld
        if out is None:
            out = torch.empty(self.shape[1:], dtype=torch.complex128, device=self.device)
        r = ctypes.c_int()
        j = ctypes.c_double()
        _check(self.lib.pcf_dmd_extrapolate(self._h, _ptr(snapshots), int(ld), int(M), float(rank_tol), _ptr(out),
                                             ctypes.byref(r), ctypes.byref(j)))
        return out, r.value, j.value

    def run(self, u, dtau, max_steps, tol=1e-10, dmd_period=100, dmd_snapshots=20, rank_tol=1e-12):
        """Descent to J < tol with optional DMD jumps; returns (steps per instance, J per instance, jumps)."""
        B = self.batch
        steps = (ctypes.c_int * B)()
        J = (ctypes.c_double * B)()
        jumps = ctypes.c_int()
        self._chk(u)
        _check(self.lib.pcf_run(self._h, _ptr(u), float(dtau), int(max_steps), float(tol), int(dmd_period),
                                int(dmd_snapshots), float(rank_tol), steps, J, ctypes.byref(jumps)))
        return list(steps), list(J), jumps.value

    def run_schedule(self, u, dtau, max_steps, tol=1e-10, snapshots=101, spacing=100, gap=0, j_start=math.inf,
                     rank_tol=1e-12, dmd=True):
        """Descent to J < tol with the DMD schedule of §6.2 (see include/pcfadj.h); returns
        (steps per instance, J per instance, jumps)."""
        B = self.batch
        steps = (ctypes.c_int * B)()
        J = (ctypes.c_double * B)()
        jumps = ctypes.c_int()
        self._chk(u)
        sc = _Schedule(snapshots, spacing, gap, j_start, rank_tol)
        _check(self.lib.pcf_run_schedule(self._h, _ptr(u), float(dtau), int(max_steps), float(tol),
                                         ctypes.byref(sc) if dmd else None, steps, J, ctypes.byref(jumps)))
        return list(steps), list(J), jumps.value

    def set_kernel_timing(self, enable):
        _check(self.lib.pcf_set_kernel_timing(self._h, 1 if enable else 0))

    def kernel_times(self):
        n = len(self.KERNEL_CLASSES)
        ms = (ctypes.c_double * n)()
        cnt = (ctypes.c_longlong * n)()
        _check(self.lib.pcf_kernel_times(self._h, ms, cnt, n))
        return {k: (ms[i], cnt[i]) for i, k in enumerate(self.KERNEL_CLASSES)}

    def plane_variant(self):
        """0 shared-memory Stockham plane kernels, 1 transforms in warp registers (FP32 form)."""
        return int(self.lib.pcf_plane_variant(self._h))

    def contraction_variant(self):
        """1 tcgen05 (tensor-memory accumulator), 0 mma.sync: the mixed form's Chebyshev transforms."""
        return int(self.lib.pcf_contraction_variant(self._h))

    def symmetric_modes(self):
        """Fourier modes per instance the per-mode kernels of a descent step process."""
        return int(self.lib.pcf_symmetric_modes(self._h))

    def solve_variant(self):
        """0 banded sweeps, 1 dense operators (single per-mode kernel), 2 dense split kernels."""
        return int(self.lib.pcf_solve_variant(self._h))

    def launches_per_step(self):
        return int(self.lib.pcf_launches_per_step(self._h))

    def split_config(self):
        """Autotuned organisation of the split per-mode kernels: dict of group sizes and mode tiles."""
        cfg = (ctypes.c_int * 4)()
        _check(self.lib.pcf_split_config(self._h, cfg))
        return {"group": cfg[0], "analysis_mode_tile": cfg[1], "synthesis_mode_tile": cfg[2], "solve_group": cfg[3]}

    def launches_per_call(self, nsteps=1):
        """Kernel launches of one descent_step call of nsteps steps."""
        return int(self.lib.pcf_launches_per_call(self._h, int(nsteps)))


class FNO:
    """Learned proposal network (see include/pcfadj.h); features/targets are float32 CUDA
    tensors [MP, S, NY, 4] with MP = Mx*Mz retained Fourier modes and NY = ny."""

    def __init__(self, MP, NY, width=32, layers=4, seed=0):
        import torch
        self.lib = load_library()
        self.MP, self.NY, self.W, self.L = MP, NY, width, layers
        h = ctypes.c_void_p()
        _check(self.lib.pcf_fno_create(MP, NY, width, layers, seed, _stream(), ctypes.byref(h)))
        self._h = h
        self.device = torch.device("cuda", torch.cuda.current_device())

    def close(self):
        if getattr(self, "_h", None):
            self.lib.pcf_fno_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def num_params(self):
        return int(self.lib.pcf_fno_num_params(self._h))

    def get_params(self):
        import numpy as np
        out = np.empty(self.num_params(), np.float32)
        _check(self.lib.pcf_fno_get_params(self._h, out.ctypes.data_as(ctypes.c_void_p)))
        return out

    def set_params(self, flat):
        import numpy as np
        flat = np.ascontiguousarray(flat, dtype=np.float32)
        assert flat.size == self.num_params()
        _check(self.lib.pcf_fno_set_params(self._h, flat.ctypes.data_as(ctypes.c_void_p)))

    def pack(self, p):
        """Oracle-style parameter dict -> flat float32 array in the library's layout."""
        import numpy as np
        parts = [p["E"], p["bE"], p["D"], p["bD"]]
        for l in range(self.L):
            parts += [p[f"R{l}"], p[f"L{l}"], p[f"b{l}"]]
        return np.concatenate([np.asarray(a, np.float64).ravel() for a in parts]).astype(np.float32)

    def unpack(self, flat):
        W, MP, F = self.W, self.MP, self.NY * 4
        shapes = [("E", (MP, W, F)), ("bE", (W,)), ("D", (MP, F, W)), ("bD", (MP, F))]
        for l in range(self.L):
            shapes += [(f"R{l}", (MP, W, W)), (f"L{l}", (W, W)), (f"b{l}", (W,))]
        out, o = {}, 0
        for k, shp in shapes:
            n = 1
            for d in shp:
                n *= d
            out[k] = flat[o:o + n].reshape(shp)
            o += n
        return out

    def forward(self, X, Y=None):
        import torch
        S = X.shape[1]
        Y = torch.empty_like(X) if Y is None else Y
        _check(self.lib.pcf_fno_forward(self._h, _ptr(X), S, _ptr(Y)))
        return Y

    def loss_grad(self, X, T):
        import torch
        g = torch.empty(self.num_params(), dtype=torch.float32, device=self.device)
        loss = ctypes.c_double()
        _check(self.lib.pcf_fno_loss_grad(self._h, _ptr(X), _ptr(T), X.shape[1], ctypes.byref(loss), _ptr(g)))
        return loss.value, g

    def train_step(self, X, T, lr):
        loss = ctypes.c_double()
        _check(self.lib.pcf_fno_train_step(self._h, _ptr(X), _ptr(T), X.shape[1], float(lr), ctypes.byref(loss)))
        return loss.value

    @staticmethod
    def unit_scale(solver):
        import torch
        MP = solver.shape[2] * solver.shape[3]
        return torch.ones((MP, solver.ny, 4), dtype=torch.float32, device=solver.device)

    @staticmethod
    def features(solver, u, scale=None, X=None):
        """Scaled features [MP, batch, NY, 4]; scale: float32 [MP, NY, 4] (default ones)."""
        import torch
        MP = solver.shape[2] * solver.shape[3]
        scale = FNO.unit_scale(solver) if scale is None else scale
        X = torch.empty((MP, solver.batch, solver.ny, 4), dtype=torch.float32, device=solver.device) if X is None else X
        _check(solver.lib.pcf_fno_features(solver._h, _ptr(u), _ptr(X), _ptr(scale)))
        return X

    def propose(self, solver, u, scale, relax_steps=0, dtau=0.01):
        """One judged proposal on every instance of ``solver``; returns (accepted, J_plain, J_proposal)."""
        B = solver.batch
        acc = (ctypes.c_int * B)()
        j0 = (ctypes.c_double * B)()
        j1 = (ctypes.c_double * B)()
        _check(self.lib.pcf_fno_propose(solver._h, self._h, _ptr(u), _ptr(scale), int(relax_steps), float(dtau),
                                        acc, j0, j1))
        return list(acc), list(j0), list(j1)
