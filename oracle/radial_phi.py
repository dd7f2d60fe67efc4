"""The paper's radial scheme for the HBE (test infrastructure only).

Sec. 2.2 reduces radially symmetric solutions to Eq. (radial),

    phi_tt - e^{-2t} (phi_rr + (2/r) phi_r) + 3 phi_t = mu^2 phi - lambda phi^3,

on 0 <= r <= R (physical units: the paper's r in (0, 1) with the factor 1/L^2
is R = L here), phi_r(0) = 0, phi(R) = 0.  This module is that scheme written
out plainly in FP64 numpy:

* nodes r_i = i dr, dr = R / n, unknowns i = 0 .. n-1 (node n is the wall);
* interior nodes: the fourth-order second difference of Sec. 2.1 for phi_rr
  and the fourth-order central first difference for phi_r (the paper states
  fourth order but prints no first-derivative stencil);
* ghosts: phi(-r) = phi(r) (the symmetry the paper uses at r = 0) and zero at
  the wall and beyond it (as for the 3D zero-Dirichlet ghosts);
* the origin: (2/r) phi_r -> 2 phi_rr(0) (L'Hospital, Sec. 2.2), so the
  operator there is 3 phi_rr(0) with the even closure the paper prints,
  (-5/2 phi_0 + 8/3 phi_1 - 1/6 phi_2) / dr^2;
* time: the textbook RK4 with four k arrays (Sec. 2.1), t_n = t0 + n dt.

It shares no code with the GPU radial kernel.  Its pins are in
tests/test_oracle_pins.py (P11): exactness on even polynomials, a linear
spherical-Bessel mode against an ODE solve, fourth-order convergence, and
agreement with the independent u = r phi solver of `radial.py`.
"""
from __future__ import annotations

from typing import Dict, List, Optional, Tuple

import numpy as np

# fourth-order weights (Sec. 2.1): second difference and first difference
_D2 = (-1.0 / 12.0, 4.0 / 3.0, -5.0 / 2.0, 4.0 / 3.0, -1.0 / 12.0)
_D1 = (1.0 / 12.0, -2.0 / 3.0, 0.0, 2.0 / 3.0, -1.0 / 12.0)


def _extend(phi: np.ndarray) -> np.ndarray:
    """phi_{-2} .. phi_{n+1}: even reflection at the origin, zeros from the wall on."""
    n = phi.shape[0]
    ext = np.zeros(n + 4)
    ext[2:n + 2] = phi
    ext[1] = phi[1] if n > 1 else 0.0
    ext[0] = phi[2] if n > 2 else 0.0
    return ext


def laplacian(phi: np.ndarray, dr: float) -> np.ndarray:
    """phi_rr + (2/r) phi_r at the nodes 0 .. n-1 (3 phi_rr at the origin)."""
    n = phi.shape[0]
    e = _extend(phi)
    d2 = sum(w * e[k:k + n] for k, w in enumerate(_D2)) / (dr * dr)
    d1 = sum(w * e[k:k + n] for k, w in enumerate(_D1)) / dr
    r = np.arange(n) * dr
    out = np.empty(n)
    out[1:] = d2[1:] + 2.0 * d1[1:] / r[1:]
    out[0] = 3.0 * (-2.5 * phi[0] + (8.0 / 3.0) * e[3] - (1.0 / 6.0) * e[4]) / (dr * dr)
    return out


def rhs(t: float, phi: np.ndarray, psi: np.ndarray, dr: float, mu: float, lam: float):
    """The first-order system (phi, psi)' = (psi, -3 psi + e^{-2t} Lap phi + mu^2 phi - lambda phi^3)."""
    return psi, -3.0 * psi + np.exp(-2.0 * t) * laplacian(phi, dr) + mu * mu * phi - lam * phi ** 3


def sign_changes(phi: np.ndarray, eps: float = 0.0) -> int:
    """Number of strict sign changes along r, ignoring nodes with |phi| <= eps;
    each one is a spherical shell where the solution changes sign (a bubble
    boundary in the sense of Sec. 1)."""
    s = np.sign(phi[np.abs(phi) > eps])
    return int(np.count_nonzero(s[1:] != s[:-1]))


def run(phi0: np.ndarray, phi1: np.ndarray, R: float, mu: float, lam: float, t0: float,
        dt: float, nsteps: int, record_every: int = 0, stop: float = 0.0, eps: float = 0.0
        ) -> Dict[str, object]:
    """Integrate one problem.  phi0, phi1: values at the n nodes r_i = i R / n.
    Every `record_every` steps (and never if 0) a record (t, max|phi|, sign
    changes) is kept.  The run ends after the first step whose phi is not
    finite (status 2) or, with stop > 0, whose max|phi| exceeds stop (status 1)."""
    phi = np.array(phi0, dtype=np.float64)
    psi = np.array(phi1, dtype=np.float64)
    n = phi.shape[0]
    dr = R / n
    recs: List[Tuple[float, float, int]] = []
    status, done = 0, 0
    for k in range(nsteps):
        t = t0 + k * dt
        k1p, k1q = rhs(t, phi, psi, dr, mu, lam)
        k2p, k2q = rhs(t + dt / 2, phi + dt / 2 * k1p, psi + dt / 2 * k1q, dr, mu, lam)
        k3p, k3q = rhs(t + dt / 2, phi + dt / 2 * k2p, psi + dt / 2 * k2q, dr, mu, lam)
        k4p, k4q = rhs(t + dt, phi + dt * k3p, psi + dt * k3q, dr, mu, lam)
        phi = phi + dt / 6.0 * (k1p + 2.0 * k2p + 2.0 * k3p + k4p)
        psi = psi + dt / 6.0 * (k1q + 2.0 * k2q + 2.0 * k3q + k4q)
        done = k + 1
        m = float(np.max(np.abs(phi)))
        if record_every and done % record_every == 0:
            recs.append((t0 + done * dt, m, sign_changes(phi, eps)))
        if not np.isfinite(m):
            status = 2
            break
        if stop > 0 and m > stop:
            status = 1
            break
    return {"phi": phi, "psi": psi, "steps": done, "status": status, "records": recs}
