"""Plain FP64 CPU oracle for the adjoint-descent hot path (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline leg may
import this package.  The CUDA library never imports, links or calls it, and the two
share no code: the oracle solves each Stokes step with a dense LU of the full
Chebyshev-tau system per Fourier mode and uses numpy's FFT, while the CUDA path uses
its own transforms and banded tau solves with an influence-matrix correction.
"""
from .pcf_oracle import PCFOracle  # noqa: F401
from . import dmd  # noqa: F401
