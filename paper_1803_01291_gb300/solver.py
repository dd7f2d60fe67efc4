"""Python front end of libhbe: `Solver` (one N^3 problem) and `Batch` (many
problems advanced together).  PyTorch supplies device memory (the fields
live in a torch-allocated workspace, so the caching allocator and
`torch.cuda.mem_get_info` see them) and the CUDA stream; every step of the
method runs in libhbe's kernels."""
from __future__ import annotations

import ctypes
from typing import List, Optional, Tuple

import numpy as np

from . import _lib
from ._lib import (BF16, DIRICHLET, FP32, FP32_PLAIN, FP64, HBEError, NONFINITE, OK, PERIODIC,
                   STOPPED)


def _torch():
    import torch
    if not torch.cuda.is_available():
        raise RuntimeError("libhbe needs a CUDA GPU; no device is visible")
    return torch


def _check(lib, status: int, ctx=None, batch=None, allow=(OK,)):
    if status in allow:
        return status
    if ctx is not None:
        msg = lib.hbe_last_error(ctx).decode()
    elif batch is not None:
        msg = lib.hbe_batch_last_error(batch).decode()
    else:
        msg = lib.hbe_status_string(status).decode()
    raise HBEError(status, msg)


def workspace_bytes(N: int, bc: int, prec: int) -> int:
    lib = _lib.load()
    out = ctypes.c_size_t()
    _check(lib, lib.hbe_workspace_bytes(N, bc, prec, ctypes.byref(out)))
    return out.value


def variants(prec: int) -> List[dict]:
    lib = _lib.load()
    out = []
    for v in range(lib.hbe_variant_count(prec)):
        info = _lib.HbeVariant()
        _check(lib, lib.hbe_variant_info(prec, v, ctypes.byref(info)))
        out.append(dict(tile_x=info.tile_x, tile_y=info.tile_y, threads=info.threads, vec=info.vec,
                        rows_per_warp=info.rows_per_warp, consumer_warps=info.consumer_warps,
                        smem=list(info.smem_bytes), ring=list(info.ring),
                        pair_tile_y=list(info.pair_tile_y), pair_threads=list(info.pair_threads),
                        pair_smem=list(info.pair_smem_bytes), pair_ring=list(info.pair_ring)))
    return out


class Solver:
    """One HBE problem: N^3 unknowns on a box of side L (Sec. 2.1 grid),
    parameters mu, lambda, zero-Dirichlet or periodic boundary, a precision
    mode (FP64, FP32 with compensated state, BF16-stored stage values, plain FP32)."""

    def __init__(self, N: int, L: float, mu: float, lam: float, bc: int = DIRICHLET,
                 prec: int = FP64, stream=None, use_torch_memory: bool = True):
        self.lib = _lib.load()
        self.N, self.L, self.mu, self.lam, self.bc, self.prec = N, L, mu, lam, bc, prec
        self._ctx = ctypes.c_void_p()
        self._ws = None
        if use_torch_memory:
            torch = _torch()
            nbytes = workspace_bytes(N, bc, prec)
            self._ws = torch.empty(nbytes + 256, dtype=torch.uint8, device="cuda")
            ptr = self._ws.data_ptr()
            ptr = (ptr + 255) // 256 * 256
            _check(self.lib, self.lib.hbe_create_in(N, L, mu, lam, bc, prec, ctypes.c_void_p(ptr),
                                                    nbytes, ctypes.byref(self._ctx)))
        else:
            _check(self.lib, self.lib.hbe_create(N, L, mu, lam, bc, prec, ctypes.byref(self._ctx)))
        if stream is None and use_torch_memory:
            stream = _torch().cuda.current_stream().cuda_stream
        if stream is not None:
            self._chk(self.lib.hbe_set_stream(self._ctx, ctypes.c_void_p(int(stream))))

    # -- plumbing
    def _chk(self, status, allow=(OK,)):
        return _check(self.lib, status, ctx=self._ctx, allow=allow)

    @property
    def handle(self):
        return self._ctx

    def close(self):
        if self._ctx:
            self.lib.hbe_destroy(self._ctx)
            self._ctx = ctypes.c_void_p()
        self._ws = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    @property
    def h(self) -> float:
        return self.L / self.N if self.bc == PERIODIC else self.L / (self.N + 1)

    # -- API
    def set_stream(self, stream: int):
        """Enqueue this problem's later work on `stream` (a cudaStream_t)."""
        self._chk(self.lib.hbe_set_stream(self._ctx, ctypes.c_void_p(int(stream))))

    def set_tuning(self, variant: int, zchunk: int = 0):
        self._chk(self.lib.hbe_set_tuning(self._ctx, variant, zchunk))

    def set_schedule(self, schedule: int):
        """0: four one-stage kernels per RK4 step; 1 (default): two fused pairs."""
        self._chk(self.lib.hbe_set_schedule(self._ctx, schedule))

    def set_stop(self, threshold: float):
        self._chk(self.lib.hbe_set_stop(self._ctx, threshold))

    def set_initial(self, phi0, phi1, t0: float = 0.0):
        """phi0, phi1: (N, N, N) float64 arrays indexed [z, y, x], host (numpy)
        or device (torch CUDA tensors)."""
        if hasattr(phi0, "is_cuda") and phi0.is_cuda:
            torch = _torch()
            a = phi0.to(torch.float64).contiguous()
            b = phi1.to(torch.float64).contiguous()
            assert a.shape == (self.N,) * 3 and b.shape == (self.N,) * 3
            self._chk(self.lib.hbe_set_initial_device(self._ctx, ctypes.c_void_p(a.data_ptr()),
                                                      ctypes.c_void_p(b.data_ptr()), t0))
            return
        a = np.ascontiguousarray(phi0, dtype=np.float64)
        b = np.ascontiguousarray(phi1, dtype=np.float64)
        assert a.shape == (self.N,) * 3 and b.shape == (self.N,) * 3
        dp = ctypes.POINTER(ctypes.c_double)
        self._chk(self.lib.hbe_set_initial(self._ctx, a.ctypes.data_as(dp), b.ctypes.data_as(dp), t0))

    def set_initial_bumps(self, bumps0, bumps1=(), t0: float = 0.0):
        """Initial data as sums of bumps A exp(-1/(1 - r^2/R^2)) evaluated on the
        device; bumps0 / bumps1: sequences of (A, R, (cx, cy, cz))."""
        def pack(bs):
            A = np.array([b[0] for b in bs], dtype=np.float64)
            R = np.array([b[1] for b in bs], dtype=np.float64)
            c = np.array([list(b[2]) for b in bs], dtype=np.float64).reshape(-1)
            return A, R, c
        dp = ctypes.POINTER(ctypes.c_double)
        A0, R0, c0 = pack(list(bumps0))
        A1, R1, c1 = pack(list(bumps1))
        ptr = lambda a: a.ctypes.data_as(dp) if a.size else None
        self._chk(self.lib.hbe_set_initial_bumps(self._ctx, len(A0), ptr(A0), ptr(R0), ptr(c0),
                                                 len(A1), ptr(A1), ptr(R1), ptr(c1), t0))

    def step(self, nsteps: int, dt: float) -> int:
        """Advance nsteps RK4 steps; returns OK, STOPPED or NONFINITE."""
        return self._chk(self.lib.hbe_step(self._ctx, int(nsteps), float(dt)),
                         allow=(OK, STOPPED, NONFINITE))

    def step_async(self, nsteps: int, dt: float):
        self._chk(self.lib.hbe_step_async(self._ctx, int(nsteps), float(dt)))

    def sync(self) -> int:
        return self._chk(self.lib.hbe_sync(self._ctx), allow=(OK, STOPPED, NONFINITE))

    def profile_stages(self, nsteps: int, dt: float):
        """Advance nsteps with per-stage CUDA-event timing; returns the mean
        milliseconds of stages 1..4."""
        out = (ctypes.c_float * 4)()
        self._chk(self.lib.hbe_profile_stages(self._ctx, int(nsteps), float(dt), out),
                  allow=(OK, STOPPED, NONFINITE))
        return [float(v) for v in out]

    def progress(self) -> Tuple[int, float]:
        n = ctypes.c_int64()
        t = ctypes.c_double()
        self._chk(self.lib.hbe_progress(self._ctx, ctypes.byref(n), ctypes.byref(t)))
        return n.value, t.value

    def read(self, psi: bool = True):
        """(phi, psi or None, t) as float64 numpy arrays [z, y, x]."""
        N = self.N
        phi = np.empty((N, N, N))
        ps = np.empty((N, N, N)) if psi else None
        t = ctypes.c_double()
        dp = ctypes.POINTER(ctypes.c_double)
        self._chk(self.lib.hbe_read(self._ctx, phi.ctypes.data_as(dp),
                                    ps.ctypes.data_as(dp) if psi else None, ctypes.byref(t)))
        return phi, ps, t.value

    @staticmethod
    def _host_field(a, N):
        if not (isinstance(a, np.ndarray) and a.dtype == np.float64 and a.shape == (N,) * 3
                and a.flags.c_contiguous):
            raise ValueError("expected a C-contiguous float64 numpy array of shape (N, N, N)")
        return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))

    def prefetch_initial(self, phi0, phi1):
        """Start copying host arrays phi0, phi1 (C-contiguous float64 (N, N, N);
        page-locked memory lets the copy overlap the steps) into the context's
        staging area and return; they become the initial data at the next
        set_initial_prefetched and must not change until then."""
        a, b = self._host_field(phi0, self.N), self._host_field(phi1, self.N)
        self._chk(self.lib.hbe_prefetch_initial(self._ctx, a, b))
        self._prefetched = (phi0, phi1)

    def set_initial_prefetched(self, t0: float = 0.0):
        self._chk(self.lib.hbe_set_initial_prefetched(self._ctx, t0))
        self._prefetched = None

    def read_async(self, phi_out, psi_out=None):
        """Start reading phi (and psi) into the given host arrays and return;
        they hold the state once read_wait() returns."""
        a = self._host_field(phi_out, self.N)
        b = self._host_field(psi_out, self.N) if psi_out is not None else None
        self._chk(self.lib.hbe_read_async(self._ctx, a, b))
        self._reading = (phi_out, psi_out)

    def read_wait(self):
        self._chk(self.lib.hbe_read_wait(self._ctx))
        self._reading = None

    def read_device(self, phi_out=None, psi_out=None):
        """State into float64 torch CUDA tensors (allocated if not given)."""
        torch = _torch()
        N = self.N
        if phi_out is None:
            phi_out = torch.empty((N, N, N), dtype=torch.float64, device="cuda")
        self._chk(self.lib.hbe_read_device(
            self._ctx, ctypes.c_void_p(phi_out.data_ptr()),
            ctypes.c_void_p(psi_out.data_ptr()) if psi_out is not None else None))
        return phi_out, psi_out

    def diag(self, eps: float = 0.0, masks: bool = False) -> dict:
        """max|phi|, finiteness, sign masks (optional) and the bubble count."""
        N = self.N
        W = (N + 31) // 32
        out = _lib.HbeDiag()
        pm = np.zeros((N, N, W), dtype=np.uint32) if masks else None
        nm = np.zeros((N, N, W), dtype=np.uint32) if masks else None
        self._chk(self.lib.hbe_diag(self._ctx, eps, ctypes.byref(out),
                                    pm.ctypes.data_as(ctypes.c_void_p) if masks else None,
                                    nm.ctypes.data_as(ctypes.c_void_p) if masks else None))
        d = dict(t=out.t, step=out.step, max_abs_phi=out.max_abs_phi, finite=bool(out.finite),
                 n_pos=out.n_pos, n_neg=out.n_neg, bubble_count=out.bubble_count)
        if masks:
            d["pos_mask"], d["neg_mask"] = pm, nm
        return d

    def analysis(self, eps: float = 0.0) -> dict:
        """Sec. 3 analysis quantities: integral of phi and phi^3, the Laplacian
        monitor e^{-2t} max|Lap phi|, and the first bubble condition's violations."""
        out = _lib.HbeAnalysis()
        self._chk(self.lib.hbe_analysis(self._ctx, eps, ctypes.byref(out)))
        return {f: getattr(out, f) for f, _ in _lib.HbeAnalysis._fields_}

    def set_monitor(self, on: bool = True):
        """Record the Laplacian monitor P(t_n) of every step's starting state
        from the stages 1+2 kernel (Sec. 3)."""
        self._chk(self.lib.hbe_set_monitor(self._ctx, int(bool(on))))

    def monitor(self, first: int, count: int):
        """(P, t) arrays of the monitor for the states before steps first ..
        first + count - 1."""
        P = np.empty(count)
        t = np.empty(count)
        dp = ctypes.POINTER(ctypes.c_double)
        self._chk(self.lib.hbe_monitor_read(self._ctx, int(first), int(count),
                                            P.ctypes.data_as(dp), t.ctypes.data_as(dp)))
        return P, t

    def save(self, path: str):
        self._chk(self.lib.hbe_save(self._ctx, path.encode()))

    def load(self, path: str):
        self._chk(self.lib.hbe_load(self._ctx, path.encode()))

    @property
    def launches(self) -> int:
        return self.lib.hbe_launch_count(self._ctx)


class Batch:
    """Continuous batching of Solvers of one precision: each run advances
    every member by up to K steps with one CUDA-graph replay (4 persistent
    stage launches per step over all members' tiles)."""

    def __init__(self, prec: int = FP32, K: int = 8, stream=None):
        self.lib = _lib.load()
        if stream is None:
            stream = _torch().cuda.current_stream().cuda_stream
        self._b = ctypes.c_void_p()
        _check(self.lib, self.lib.hbe_batch_create(prec, K, ctypes.c_void_p(int(stream)),
                                                   ctypes.byref(self._b)))
        self._members = {}
        self.K = K

    def _chk(self, status):
        return _check(self.lib, status, batch=self._b)

    def add(self, solver: Solver, nsteps: int, dt: float):
        self._chk(self.lib.hbe_batch_add(self._b, solver.handle, int(nsteps), float(dt)))
        self._members[solver.handle.value] = solver

    def remove(self, solver: Solver):
        self._chk(self.lib.hbe_batch_remove(self._b, solver.handle))
        self._members.pop(solver.handle.value, None)

    def run(self) -> List[Solver]:
        """One run of up to K steps for every member; returns the members that
        finished (reached their step count or stopped)."""
        self.launch()
        return self.collect()

    def launch(self):
        """Enqueue one run and return at once (collect() waits for it)."""
        self._chk(self.lib.hbe_batch_launch(self._b))

    def collect(self) -> List[Solver]:
        """Wait for the run in flight and return the members that finished."""
        cap = max(1, len(self._members))
        arr = (ctypes.c_void_p * cap)()
        n = ctypes.c_int()
        self._chk(self.lib.hbe_batch_collect(self._b, arr, cap, ctypes.byref(n)))
        done = [self._members.pop(arr[i]) for i in range(n.value)]
        return done

    def __len__(self):
        return self.lib.hbe_batch_size(self._b)

    @property
    def launches(self) -> int:
        return self.lib.hbe_batch_launch_count(self._b)

    def close(self):
        if self._b:
            self.lib.hbe_batch_destroy(self._b)
            self._b = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
