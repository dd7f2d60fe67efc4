"""z-slab decomposition of one N^3 grid.

The fourth-order stencil of Sec. 2.1 reaches two planes in each direction,
so a grid split along z into k slabs advances each slab with the same stage
kernels once two planes of every neighbour are present: after the stages
1+2 kernel the neighbours' G1, G2 planes, after the stages 3+4 kernel their
new phi, psi planes.  `plan` gives the slab sizes and the list of 2-plane
transfers (computed by libhbe, `hbe_slab_plan`); `SlabSolver` runs k virtual
slabs on one GPU, the halo transfers being device copies into each
receiving slab's own buffers (bitwise the undivided grid's result);
`exchange_halos` carries out the same plan between ranks of a
torch.distributed process group, one slab per rank.
"""
from __future__ import annotations

import ctypes
from typing import List, Tuple

import numpy as np

from . import _lib
from .solver import _check, _torch

HALO = 2  # stored halo planes on each side of a slab


def plan(N: int, k: int, periodic: bool) -> Tuple[List[int], List[Tuple[int, int, int, int]]]:
    """(planes of each slab, transfers (src slab, dst slab, src stored plane,
    dst stored plane), 2 planes each).  Slab i stores its planes at stored
    planes 2 .. nz_i + 1, with halo planes 0, 1 and nz_i + 2, nz_i + 3."""
    lib = _lib.load()
    nz = (ctypes.c_int32 * max(k, 1))()
    n = lib.hbe_slab_plan(N, k, int(bool(periodic)), nz, None, 0)
    if n < 0:
        raise ValueError(f"no slab plan for N={N}, k={k} (need k >= 1 and N >= 2k)")
    cp = (ctypes.c_int32 * (4 * max(n, 1)))()
    lib.hbe_slab_plan(N, k, int(bool(periodic)), nz, cp, n)
    copies = [tuple(int(v) for v in cp[4 * i:4 * i + 4]) for i in range(n)]
    return [int(v) for v in nz[:k]], copies


def exchange_halos(local, rank: int, copies, group=None):
    """Carry out the transfers of `copies` that involve `rank`: `local` is the
    rank's stored block (nz + 4 planes along dim 0, halos included).  Sends
    and receives are point to point (tag = transfer index); a transfer from a
    rank to itself (one periodic slab) is a local copy."""
    import torch.distributed as dist
    reqs, recv = [], []
    for tag, (src, dst, sp, dp) in enumerate(copies):
        if src == rank and dst == rank:
            local[dp:dp + HALO] = local[sp:sp + HALO].clone()
        elif src == rank:
            reqs.append(dist.isend(local[sp:sp + HALO].contiguous(), dst, group=group, tag=tag))
        elif dst == rank:
            buf = local.new_empty(local[dp:dp + HALO].shape)
            reqs.append(dist.irecv(buf, src, group=group, tag=tag))
            recv.append((dp, buf))
    for r in reqs:
        r.wait()
    for dp, buf in recv:
        local[dp:dp + HALO] = buf


class SlabSolver:
    """One N^3 problem advanced as k z-slabs on the current GPU (same
    arguments as Solver, plus k).  Initial data and results are whole-grid
    float64 arrays [z, y, x]; numpy arrays go through the device."""

    def __init__(self, N: int, L: float, mu: float, lam: float, bc: int = _lib.DIRICHLET,
                 prec: int = _lib.FP64, k: int = 2, stream=None):
        torch = _torch()
        self.lib = _lib.load()
        self.N, self.k = N, k
        if stream is None:
            stream = torch.cuda.current_stream().cuda_stream
        self._s = ctypes.c_void_p()
        _check(self.lib, self.lib.hbe_slabs_create(N, L, mu, lam, bc, prec, k,
                                                   ctypes.c_void_p(int(stream)),
                                                   ctypes.byref(self._s)))

    def _chk(self, status, allow=(_lib.OK,)):
        if status in allow:
            return status
        raise _lib.HBEError(status, self.lib.hbe_slabs_last_error(self._s).decode())

    def set_initial(self, phi0, phi1, t0: float = 0.0):
        torch = _torch()
        a = torch.as_tensor(np.asarray(phi0) if not hasattr(phi0, "is_cuda") else phi0)
        b = torch.as_tensor(np.asarray(phi1) if not hasattr(phi1, "is_cuda") else phi1)
        a = a.to(device="cuda", dtype=torch.float64).contiguous()
        b = b.to(device="cuda", dtype=torch.float64).contiguous()
        assert a.shape == (self.N,) * 3 and b.shape == (self.N,) * 3
        torch.cuda.synchronize()
        self._chk(self.lib.hbe_slabs_set_initial_device(self._s, ctypes.c_void_p(a.data_ptr()),
                                                        ctypes.c_void_p(b.data_ptr()), t0))

    def step(self, nsteps: int, dt: float) -> int:
        return self._chk(self.lib.hbe_slabs_step(self._s, int(nsteps), float(dt)),
                         allow=(_lib.OK, _lib.NONFINITE))

    def read(self):
        """(phi, psi, t) of the whole grid as float64 numpy arrays."""
        torch = _torch()
        N = self.N
        phi = torch.empty((N, N, N), dtype=torch.float64, device="cuda")
        psi = torch.empty_like(phi)
        t = ctypes.c_double()
        self._chk(self.lib.hbe_slabs_read_device(self._s, ctypes.c_void_p(phi.data_ptr()),
                                                 ctypes.c_void_p(psi.data_ptr()),
                                                 ctypes.byref(t)))
        return phi.cpu().numpy(), psi.cpu().numpy(), t.value

    def close(self):
        if self._s:
            self.lib.hbe_slabs_destroy(self._s)
            self._s = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()
