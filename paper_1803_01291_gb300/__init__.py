"""GB300-native solver for the Higgs boson equation in de Sitter spacetime
(arXiv:1803.01291, Sec. 2.1: FD4 in space, classic RK4 in time).

    from paper_1803_01291_gb300 import Solver, FP32, DIRICHLET
    s = Solver(N=256, L=20.0, mu=2 ** 0.5, lam=1.0, bc=DIRICHLET, prec=FP32)
    s.set_initial(phi0, phi1)          # (N, N, N) float64, [z, y, x]
    s.step(257, dt)                    # RK4 steps on the GPU
    phi, psi, t = s.read()
    s.diag()                           # max|phi|, sign masks, bubble count

The CUDA library (libhbe.so, C ABI in include/hbe.h) does all the work; this
package only marshals arguments.  `serve` holds the continuous-batching
server and `autotune` the tile/z-chunk tuner.
"""
from ._lib import (BF16, DIRICHLET, FP32, FP32_PLAIN, FP64, HBEError, NONFINITE, OK, PERIODIC,
                   PREC_NAMES, STOPPED)
from .solver import Batch, Solver, variants, workspace_bytes

__all__ = ["Solver", "Batch", "variants", "workspace_bytes", "HBEError", "FP64", "FP32", "BF16",
           "FP32_PLAIN", "DIRICHLET", "PERIODIC", "OK", "STOPPED", "NONFINITE", "PREC_NAMES"]
