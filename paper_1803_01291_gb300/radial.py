"""Batched radial solver (Sec. 2.2, Eq. radial) on the GPU.

    from paper_1803_01291_gb300 import radial
    out = radial.run(phi0, phi1, R=5.0, mu=mus, lam=lams, t0=0.0, dt=1e-3, nsteps=3000,
                     record_every=100, stop=1e6)
    out.phi, out.psi        # [batch, n] float64 device tensors after the last step
    out.records             # [batch, nsteps // record_every, 3]: t, max|phi|, sign changes
    out.steps, out.status   # steps taken; 0 done, 1 stopped at the threshold, 2 not finite

phi0, phi1 hold each problem's values at the nodes r_i = i R / n (i = 0 .. n-1;
the wall r = R carries phi = 0).  The whole integration of every problem runs
in one launch of libhbe's radial kernel (one CTA per problem); this module only
allocates the device arrays and marshals the call.
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass
from typing import Optional, Sequence, Union

import numpy as np

from . import _lib
from ._lib import FP32, FP64


def _torch():
    import torch
    if not torch.cuda.is_available():
        raise RuntimeError("the radial solver needs a CUDA device (there is no CPU fallback)")
    return torch


@dataclass
class RadialResult:
    phi: "object"
    psi: "object"
    records: Optional["object"]
    steps: "object"
    status: "object"


def max_n(prec: int = FP64) -> int:
    return int(_lib.load().hbe_radial_max_n(prec))


def run(phi0, phi1, R: float, mu: Union[float, Sequence[float]], lam: Union[float, Sequence[float]],
        t0: float, dt: float, nsteps: int, prec: int = FP64, record_every: int = 0,
        stop: float = 0.0, eps: float = 0.0, stream=None) -> RadialResult:
    """Integrate every row of phi0 / phi1 ([batch, n], host or device, any float
    dtype; converted to float64 on the device) for nsteps RK4 steps.  mu and lam
    are one value per problem (or one for all).  Returns after the work is
    enqueued on `stream` (default: torch's current stream); reading the result
    tensors from torch on that stream orders after it."""
    torch = _torch()
    lib = _lib.load()
    dev = torch.device("cuda", torch.cuda.current_device())
    a = torch.as_tensor(phi0, dtype=torch.float64, device=dev).contiguous()
    b = torch.as_tensor(phi1, dtype=torch.float64, device=dev).contiguous()
    if a.dim() == 1:
        a, b = a[None], b[None]
    if a.shape != b.shape or a.dim() != 2:
        raise ValueError("phi0 and phi1 must both be [batch, n]")
    B, n = a.shape
    m = torch.as_tensor(np.broadcast_to(np.asarray(mu, dtype=np.float64), (B,)).copy(), device=dev)
    l = torch.as_tensor(np.broadcast_to(np.asarray(lam, dtype=np.float64), (B,)).copy(), device=dev)
    phi = torch.empty_like(a)
    psi = torch.empty_like(a)
    nrec = nsteps // record_every if record_every > 0 else 0
    rec = torch.empty((B, nrec, 3), dtype=torch.float64, device=dev) if nrec > 0 else None
    steps = torch.empty(B, dtype=torch.int64, device=dev)
    status = torch.empty(B, dtype=torch.int32, device=dev)
    st = stream if stream is not None else torch.cuda.current_stream()
    vp = ctypes.c_void_p
    r = lib.hbe_radial_run(B, n, R, vp(m.data_ptr()), vp(l.data_ptr()), vp(a.data_ptr()),
                           vp(b.data_ptr()), t0, dt, nsteps, prec, record_every, stop, eps,
                           vp(phi.data_ptr()), vp(psi.data_ptr()),
                           vp(rec.data_ptr()) if rec is not None else None,
                           vp(steps.data_ptr()), vp(status.data_ptr()), vp(st.cuda_stream))
    if r != _lib.OK:
        raise _lib.HBEError(r, "hbe_radial_run rejected its arguments" if r == _lib.EINVAL
                            else "hbe_radial_run launch failed")
    # keep the inputs alive until the kernel has read them
    for t in (a, b, m, l):
        t.record_stream(st)
    return RadialResult(phi, psi, rec, steps, status)
