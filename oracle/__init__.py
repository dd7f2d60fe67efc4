"""CPU oracle for the 3D Higgs boson equation (test infrastructure only).

Only the tests, `__graft_entry__.smoke()` and the CPU-baseline leg of `bench.py`
may import this package.  The product library (`paper_1803_01291_gb300`) never
imports it and has no CPU fallback.

`hbe_oracle.c` is the plain FP64 restatement of Sec. 2.1 of the paper (FD4
Laplacian, Eq. (rhs), textbook RK4); this module compiles it with gcc on first
use and wraps it with ctypes.  `radial.py` holds the 1D u = r*phi solver used as
an independent pin; `radial_phi.py` is the paper's own radial scheme (Sec. 2.2,
phi form with the L'Hospital closure at the origin), the oracle of the batched
radial GPU solver.

Parity: every function here is pinned by tests/test_oracle_pins.py against
closed forms, library ODE solvers, invariants or brute force.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import sys
import threading
from typing import Optional, Tuple

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hbe_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle_hbe.so")
_lock = threading.Lock()
_lib = None

DIRICHLET = 0
PERIODIC = 1


def build(force: bool = False) -> str:
    """Compile hbe_oracle.c into liboracle_hbe.so (gcc, OpenMP, no FP contraction)."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
               "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        build()
        lib = ctypes.CDLL(_LIB_PATH)
        dp = ctypes.POINTER(ctypes.c_double)
        lib.oracle_grid_spacing.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_int]
        lib.oracle_grid_spacing.restype = ctypes.c_double
        lib.oracle_run.argtypes = [dp, dp, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                   ctypes.c_double, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                   ctypes.c_int64, ctypes.c_double, ctypes.c_int]
        lib.oracle_run.restype = ctypes.c_int64
        lib.oracle_run_box.argtypes = [dp, dp, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                       ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                       ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                       ctypes.c_int64, ctypes.c_double, ctypes.c_int]
        lib.oracle_run_box.restype = ctypes.c_int64
        lib.oracle_laplacian.argtypes = [dp, dp, ctypes.c_int, ctypes.c_double, ctypes.c_int,
                                         ctypes.c_int]
        lib.oracle_laplacian.restype = None
        lib.oracle_rhs.argtypes = [ctypes.c_double, dp, dp, dp, dp, ctypes.c_int, ctypes.c_double,
                                   ctypes.c_double, ctypes.c_double, ctypes.c_int]
        lib.oracle_rhs.restype = ctypes.c_int
        lib.oracle_max_abs.argtypes = [dp, ctypes.c_int, ctypes.POINTER(ctypes.c_int)]
        lib.oracle_max_abs.restype = ctypes.c_double
        u32p = ctypes.POINTER(ctypes.c_uint32)
        i64p = ctypes.POINTER(ctypes.c_int64)
        lib.oracle_diag.argtypes = [dp, ctypes.c_int, ctypes.c_int, ctypes.c_double, dp,
                                    ctypes.POINTER(ctypes.c_int), i64p, i64p, i64p, u32p, u32p]
        lib.oracle_diag.restype = ctypes.c_int
        lib.oracle_max_threads.argtypes = []
        lib.oracle_max_threads.restype = ctypes.c_int
        _lib = lib
        return lib


def _dp(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def grid_spacing(N: int, L: float, bc: int) -> float:
    return _load().oracle_grid_spacing(N, L, bc)


def max_threads() -> int:
    return _load().oracle_max_threads()


def run(phi0: np.ndarray, phi1: np.ndarray, L: float, mu: float, lam: float, bc: int,
        t0: float, dt: float, nsteps: int, stop_threshold: float = 0.0,
        nthreads: int = 0) -> Tuple[np.ndarray, np.ndarray, int]:
    """RK4 + FD4 solve (Sec. 2.1) from (phi0, phi1) at t0; returns (phi, psi, steps)."""
    N = phi0.shape[0]
    assert phi0.shape == (N, N, N) and phi1.shape == (N, N, N)
    phi = np.array(phi0, dtype=np.float64, order="C", copy=True)
    psi = np.array(phi1, dtype=np.float64, order="C", copy=True)
    n = _load().oracle_run(_dp(phi), _dp(psi), N, L, mu, lam, bc, t0, dt, int(nsteps),
                           stop_threshold, int(nthreads))
    if n < 0:
        raise MemoryError("oracle_run: allocation failed")
    return phi, psi, int(n)


def laplacian(u: np.ndarray, h: float, bc: int, nthreads: int = 0) -> np.ndarray:
    """FD4 13-point Laplacian of Sec. 2.1 (ghosts 0 or periodic wrap)."""
    u = np.ascontiguousarray(u, dtype=np.float64)
    out = np.empty_like(u)
    _load().oracle_laplacian(_dp(u), _dp(out), u.shape[0], h, bc, int(nthreads))
    return out


def rhs(t: float, v1: np.ndarray, v2: np.ndarray, L: float, mu: float, lam: float,
        bc: int) -> Tuple[np.ndarray, np.ndarray]:
    """f(t, v) of Eq. (rhs)."""
    v1 = np.ascontiguousarray(v1, dtype=np.float64)
    v2 = np.ascontiguousarray(v2, dtype=np.float64)
    f1 = np.empty_like(v1)
    f2 = np.empty_like(v1)
    if _load().oracle_rhs(t, _dp(v1), _dp(v2), _dp(f1), _dp(f2), v1.shape[0], L, mu, lam, bc):
        raise MemoryError("oracle_rhs: allocation failed")
    return f1, f2


def diag(phi: np.ndarray, bc: int, eps: float = 0.0, masks: bool = True) -> dict:
    """max|phi|, finiteness, sign masks and bubble count (Sec. 1 definition)."""
    phi = np.ascontiguousarray(phi, dtype=np.float64)
    N = phi.shape[0]
    W = (N + 31) // 32
    mx = ctypes.c_double()
    fin = ctypes.c_int()
    npos, nneg, nb = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
    pm = np.zeros((N, N, W), dtype=np.uint32) if masks else None
    nm = np.zeros((N, N, W), dtype=np.uint32) if masks else None
    u32p = ctypes.POINTER(ctypes.c_uint32)
    rc = _load().oracle_diag(_dp(phi), N, bc, eps, ctypes.byref(mx), ctypes.byref(fin),
                             ctypes.byref(npos), ctypes.byref(nneg), ctypes.byref(nb),
                             pm.ctypes.data_as(u32p) if masks else None,
                             nm.ctypes.data_as(u32p) if masks else None)
    if rc:
        raise MemoryError("oracle_diag: allocation failed")
    out = dict(max_abs_phi=mx.value, finite=bool(fin.value), n_pos=npos.value,
               n_neg=nneg.value, bubble_count=nb.value)
    if masks:
        out["pos_mask"] = pm
        out["neg_mask"] = nm
    return out


def run_box(phi0: np.ndarray, phi1: np.ndarray, h: float, mu: float, lam: float, bc: int,
            t0: float, dt: float, nsteps: int, nthreads: int = 0) -> Tuple[np.ndarray, np.ndarray]:
    """The same scheme on an (nz, ny, nx) box of unknowns with spacing h."""
    nz, ny, nx = phi0.shape
    phi = np.array(phi0, dtype=np.float64, order="C", copy=True)
    psi = np.array(phi1, dtype=np.float64, order="C", copy=True)
    n = _load().oracle_run_box(_dp(phi), _dp(psi), nx, ny, nz, h, mu, lam, bc, t0, dt,
                               int(nsteps), 0.0, int(nthreads))
    if n < 0:
        raise MemoryError("oracle_run_box: allocation failed")
    return phi, psi


def window_values(phi0: np.ndarray, phi1: np.ndarray, L: float, mu: float, lam: float,
                  bc: int, t0: float, dt: float, nsteps: int, points) -> np.ndarray:
    """Oracle (phi, psi) after `nsteps` at selected nodes (z, y, x), one at a time.

    One RK4 step moves information at most 8 nodes along an axis (4 stages of a
    radius-2 stencil), so the value at a node after n steps depends only on the
    input within r = 8n nodes of it.  Each point is computed by running the plain
    oracle on the window of nodes within r of it:
      * zero-Dirichlet: the window is clipped to the grid, so where it meets the
        wall its own zero ghosts are the grid's; elsewhere its edge lies more than
        r nodes from the point and cannot reach it;
      * periodic: indices wrap and the window (solved with zero ghosts) again has
        its edge more than r nodes away.
    The arithmetic at the point is then the full-grid oracle's, operation by
    operation."""
    N = phi0.shape[0]
    r = 8 * nsteps
    h = grid_spacing(N, L, bc)
    out = np.empty((len(points), 2))
    for n, pt in enumerate(points):
        idx, centre = [], []
        for c in pt:
            if bc == PERIODIC:
                a = np.mod(np.arange(c - r, c + r + 1), N)
                centre.append(r)
            else:
                lo, hi = max(0, c - r), min(N - 1, c + r)
                a = np.arange(lo, hi + 1)
                centre.append(c - lo)
            idx.append(a)
        w0 = np.ascontiguousarray(phi0[np.ix_(*idx)])
        w1 = np.ascontiguousarray(phi1[np.ix_(*idx)])
        a, b = run_box(w0, w1, h, mu, lam, DIRICHLET, t0, dt, nsteps)
        out[n, 0] = a[tuple(centre)]
        out[n, 1] = b[tuple(centre)]
    return out
