"""1D radial solver for the HBE (test infrastructure only).

For radially symmetric data the paper reduces the problem to Eq. (radial),
phi_tt - e^{-2t} (phi_rr + 2 phi_r / r) + 3 phi_t = mu^2 phi - lambda phi^3,
and reports that radial and 3D runs agree (Sec. 2.2).  This module solves the
equivalent form for u = r phi (phi_rr + 2 phi_r / r = u_rr / r):

    u_tt - e^{-2t} u_rr + 3 u_t = mu^2 u - lambda u^3 / r^2,   u(0, t) = 0,

on r in [0, R] with u(R, t) = 0, FD4 in r (Sec. 2.1 stencil), ghosts at r < 0
by odd reflection u(-r) = -u(r), and classic RK4 in time.  It is a different
discretisation from the 3D oracle (one space dimension, another unknown, a
fine grid of its own), so agreement to O(h^4) pins the 3D assembly: all three
axes present, the e^{-2t} factor, the damping and the cubic term.
"""
from __future__ import annotations

import numpy as np


def _d2(u: np.ndarray, dr: float) -> np.ndarray:
    """FD4 second difference on nodes r_i = i dr (i = 0..M), odd ghosts at the
    origin and zero ghosts beyond r_M."""
    M = u.shape[0] - 1
    ext = np.zeros(M + 5)
    ext[2:M + 3] = u
    ext[1] = -u[1]
    ext[0] = -u[2]
    c = ext[2:M + 3]
    return (-1.0 / 12.0 * (ext[0:M + 1] + ext[4:M + 5]) + 4.0 / 3.0 * (ext[1:M + 2] + ext[3:M + 4])
            - 5.0 / 2.0 * c) / (dr * dr)


def solve(phi0_r, phi1_r, R: float, M: int, mu: float, lam: float, T: float,
          dt: float):
    """Integrate to time T (nsteps = round(T / dt)).  phi0_r, phi1_r are callables of r.
    Returns (r, phi(r, T)) on the nodes r_i = i R / M, i = 1..M-1 (phi = u / r)."""
    dr = R / M
    r = np.arange(M + 1) * dr
    u = r * phi0_r(r)
    v = r * phi1_r(r)
    u[0] = v[0] = 0.0
    u[M] = v[M] = 0.0
    rr = r.copy()
    rr[0] = 1.0  # u_0 = 0, so u^3 / r^2 at the origin is 0 whatever is used here
    mu2 = mu * mu

    def f(t, u, v):
        a = -3.0 * v + np.exp(-2.0 * t) * _d2(u, dr) + mu2 * u - lam * u ** 3 / (rr * rr)
        a[0] = 0.0
        a[M] = 0.0
        vv = v.copy()
        vv[0] = 0.0
        vv[M] = 0.0
        return vv, a

    nsteps = int(round(T / dt))
    for n in range(nsteps):
        t = n * dt
        k1u, k1v = f(t, u, v)
        k2u, k2v = f(t + dt / 2, u + dt / 2 * k1u, v + dt / 2 * k1v)
        k3u, k3v = f(t + dt / 2, u + dt / 2 * k2u, v + dt / 2 * k2v)
        k4u, k4v = f(t + dt, u + dt * k3u, v + dt * k3v)
        u = u + dt * (k1u + 2 * k2u + 2 * k3u + k4u) / 6.0
        v = v + dt * (k1v + 2 * k2v + 2 * k3v + k4v) / 6.0
    return r[1:M], u[1:M] / r[1:M]
