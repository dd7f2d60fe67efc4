"""Seeded synthetic initial data for the 3D Higgs boson equation (HBE).

This module is shared by the CPU oracle tests and the CUDA path.  It holds no
step of the numerical method (no stencil, no time stepping): it only samples
initial data phi0, phi1 on the grid nodes and draws seeded random workloads.

Grid convention (the node layout of the rescaled problem, Sec. 2.1 of the
paper, with N = number of unknowns per axis):

* zero-Dirichlet: h = L / (N + 1); node i sits at x_i = (i - (N - 1)/2) h,
  i = 0..N-1, so the nodes are the interior nodes of a box of side L centred
  at 0 and the boundary nodes (x = +-L/2) carry phi = 0.
* periodic: h = L / N; node i sits at x_i = (i - N/2) h, i = 0..N-1.

Both forms are written as (index - centre) * h so that the node set is
symmetric about 0 bit for bit (x_{N-1-i} == -x_i for Dirichlet).

Arrays are float64, shape (N, N, N), indexed [z, y, x] (x fastest in memory).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import List, Sequence, Tuple

import numpy as np

DIRICHLET = 0
PERIODIC = 1


def grid_spacing(N: int, L: float, bc: int) -> float:
    """h of the uniform grid (Sec. 2.1: delta x = 1/n on the unit box, i.e.
    L/n in physical units; the n - 1 interior nodes are the unknowns)."""
    if bc == DIRICHLET:
        return L / (N + 1)
    if bc == PERIODIC:
        return L / N
    raise ValueError(f"unknown boundary kind {bc}")


def grid_coords(N: int, L: float, bc: int) -> np.ndarray:
    """1D node coordinates, symmetric about 0 (see module docstring)."""
    h = grid_spacing(N, L, bc)
    i = np.arange(N, dtype=np.float64)
    centre = (N - 1) / 2.0 if bc == DIRICHLET else N / 2.0
    return (i - centre) * h


def _r2(N: int, L: float, bc: int, center: Sequence[float]) -> np.ndarray:
    x = grid_coords(N, L, bc)
    dz = (x - center[2])[:, None, None]
    dy = (x - center[1])[None, :, None]
    dx = (x - center[0])[None, None, :]
    return dx * dx + dy * dy + dz * dz


def bump_into(out: np.ndarray, L: float, bc: int, A: float, R: float,
              center: Sequence[float] = (0.0, 0.0, 0.0)) -> np.ndarray:
    """Add A * exp(-1 / (1 - r^2/R^2)) (r < R; 0 outside) to `out` (N^3, [z, y, x]).
    Only nodes inside the support's bounding box are touched."""
    N = out.shape[0]
    x = grid_coords(N, L, bc)
    sl = []
    for c in (center[2], center[1], center[0]):
        idx = np.nonzero(np.abs(x - c) < R)[0]
        if idx.size == 0:
            return out
        sl.append(slice(int(idx[0]), int(idx[-1]) + 1))
    dz = (x[sl[0]] - center[2])[:, None, None]
    dy = (x[sl[1]] - center[1])[None, :, None]
    dx = (x[sl[2]] - center[0])[None, None, :]
    r2 = dx * dx + dy * dy + dz * dz
    sub = np.zeros_like(r2)
    inside = r2 < R * R
    s = 1.0 - r2[inside] / (R * R)
    sub[inside] = A * np.exp(-1.0 / s)
    out[tuple(sl)] += sub
    return out


def bump(N: int, L: float, bc: int, A: float, R: float,
         center: Sequence[float] = (0.0, 0.0, 0.0)) -> np.ndarray:
    """A * exp(-1 / (1 - r^2/R^2)) for r < R, else 0 (peak A/e at r = 0).

    This is the normalisation used for the benchmark workloads (box [-L/2, L/2]^3,
    physical radius R)."""
    return bump_into(np.zeros((N, N, N)), L, bc, A, R, center)


def bump_paper(N: int, L: float, bc: int, C_unit: Sequence[float], R_unit: float,
               A: float = 1.0) -> np.ndarray:
    """The paper's bump B(x; C, R) = exp(1/R^2 - 1/(R^2 - |x - C|^2)) inside the
    ball, 0 outside (Eq. bump, peak 1), in unit-box coordinates: the unit box
    [0, 1]^3 is mapped onto [-L/2, L/2]^3, so x_unit = x / L + 1/2."""
    x = grid_coords(N, L, bc) / L + 0.5
    dz = (x - C_unit[2])[:, None, None]
    dy = (x - C_unit[1])[None, :, None]
    dx = (x - C_unit[0])[None, None, :]
    r2 = dx * dx + dy * dy + dz * dz
    out = np.zeros_like(r2)
    inside = r2 < R_unit * R_unit
    out[inside] = A * np.exp(1.0 / (R_unit * R_unit) - 1.0 / (R_unit * R_unit - r2[inside]))
    return out


def gaussian(N: int, L: float, bc: int, A: float, center: Sequence[float], w: float) -> np.ndarray:
    """A * exp(-|x - c|^2 / (2 w^2)), w the standard deviation."""
    return A * np.exp(-_r2(N, L, bc, center) / (2.0 * w * w))


def gaussian_sum(N: int, L: float, bc: int, rng: np.random.Generator, count: int,
                 amp: Tuple[float, float], cen: Tuple[float, float],
                 width: Tuple[float, float]) -> np.ndarray:
    """Sum of `count` Gaussians; draw order: all amplitudes, all centres
    (count x 3), all widths, each uniform on the given interval."""
    amps = rng.uniform(amp[0], amp[1], size=count)
    cens = rng.uniform(cen[0], cen[1], size=(count, 3))
    wids = rng.uniform(width[0], width[1], size=count)
    out = np.zeros((N, N, N))
    for a, c, w in zip(amps, cens, wids):
        out += gaussian(N, L, bc, a, c, w)
    return out


def plane_wave(N: int, L: float, m: Sequence[int], amp: float = 1.0) -> np.ndarray:
    """amp * cos(k . x), k = 2 pi m / L, on the periodic grid."""
    x = grid_coords(N, L, PERIODIC)
    k = [2.0 * math.pi * mi / L for mi in m]
    ph = (k[2] * x)[:, None, None] + (k[1] * x)[None, :, None] + (k[0] * x)[None, None, :]
    return amp * np.cos(ph)


def grf(N: int, L: float, seed: int, corr_len: float = 2.0) -> np.ndarray:
    """Band-limited Gaussian random field with unit sample std on the periodic grid.

    White noise N(0, 1) (PCG64, `default_rng(seed)`), filtered in Fourier space by
    H(k) = exp(-|k|^2 corr_len^2 / 4) (covariance proportional to
    exp(-r^2 / (2 corr_len^2))), modes with |k| >= k_Nyquist / 2 set to zero, then
    the sample mean removed and the sample std scaled to 1."""
    rng = np.random.default_rng(seed)
    noise = rng.standard_normal((N, N, N))
    h = L / N
    kz = 2.0 * math.pi * np.fft.fftfreq(N, d=h)
    kx = 2.0 * math.pi * np.fft.rfftfreq(N, d=h)
    spec = np.fft.rfftn(noise)
    del noise
    k_nyq = math.pi / h
    for iz in range(N):
        k2 = kz[iz] ** 2 + kz[:, None] ** 2 + kx[None, :] ** 2
        filt = np.exp(-k2 * corr_len * corr_len / 4.0)
        filt[k2 >= (k_nyq / 2.0) ** 2] = 0.0
        spec[iz] *= filt
    field = np.fft.irfftn(spec, s=(N, N, N), axes=(0, 1, 2))
    field -= field.mean()
    field /= field.std()
    return field


# ----------------------------------------------------------------------------
# Benchmark workloads (sizes and laws of the five benchmark configurations)
# ----------------------------------------------------------------------------

@dataclass
class Problem:
    """One HBE initial-value problem on an N^3 grid."""
    N: int
    L: float
    mu: float
    lam: float
    bc: int
    phi0: np.ndarray
    phi1: np.ndarray
    T: float
    dt: float
    nsteps: int
    name: str = ""


def steps_for(T: float, h: float) -> Tuple[int, float]:
    """nsteps = ceil(T / (h/4) - 1e-12), dt = T / nsteps (dt <= h/4)."""
    n = int(math.ceil(T / (h / 4.0) - 1e-12))
    return n, T / n


def radial_bump_problem(N: int = 64) -> Problem:
    """N^3 on [-5, 5]^3, zero-Dirichlet, mu = lambda = 1,
    phi0 = 1.5 exp(-1/(1 - r^2/9)), phi1 = 0, t in [0, 2], dt = h/4."""
    L = 10.0
    h = grid_spacing(N, L, DIRICHLET)
    n, dt = steps_for(2.0, h)
    return Problem(N, L, 1.0, 1.0, DIRICHLET, bump(N, L, DIRICHLET, 1.5, 3.0),
                   np.zeros((N, N, N)), 2.0, dt, n, f"radial-bump-{N}")


def gaussians_problem(N: int = 256, seed: int = 0) -> Problem:
    """N^3 on [-10, 10]^3, zero-Dirichlet, mu = sqrt(2), lambda = 1; phi0 = 8 Gaussians
    (amp U[-2,2], centre U[-6,6]^3, width U[.5,2]), phi1 = 4 Gaussians (amp U[-.5,.5]);
    t in [0, 5], dt <= h/4."""
    L = 20.0
    rng = np.random.default_rng(seed)
    phi0 = gaussian_sum(N, L, DIRICHLET, rng, 8, (-2.0, 2.0), (-6.0, 6.0), (0.5, 2.0))
    phi1 = gaussian_sum(N, L, DIRICHLET, rng, 4, (-0.5, 0.5), (-6.0, 6.0), (0.5, 2.0))
    h = grid_spacing(N, L, DIRICHLET)
    n, dt = steps_for(5.0, h)
    return Problem(N, L, math.sqrt(2.0), 1.0, DIRICHLET, phi0, phi1, 5.0, dt, n,
                   f"gaussians-{N}-seed{seed}")


def grf_problem(N: int = 512, lam: float = 1.0, seed: int = 0) -> Problem:
    """N^3 on [-20, 20]^3, periodic, mu = 1, phi0 = band-limited GRF (std 1,
    correlation length 2), phi1 = 0, t in [0, 6], dt <= h/4."""
    L = 40.0
    h = grid_spacing(N, L, PERIODIC)
    n, dt = steps_for(6.0, h)
    return Problem(N, L, 1.0, lam, PERIODIC, grf(N, L, seed), np.zeros((N, N, N)), 6.0, dt, n,
                   f"grf-{N}-lam{lam}-seed{seed}")


def blowup_problem(N: int = 1024) -> Problem:
    """N^3 on [-10, 10]^3, zero-Dirichlet, mu = 1, lambda = -1 (focusing),
    phi0 = 3 exp(-1/(1 - r^2/16)), phi1 = 0, dt = h/4, horizon cap T = 10."""
    L = 20.0
    h = grid_spacing(N, L, DIRICHLET)
    dt = h / 4.0
    return Problem(N, L, 1.0, -1.0, DIRICHLET, bump(N, L, DIRICHLET, 3.0, 4.0),
                   np.zeros((N, N, N)), 10.0, dt, int(math.ceil(10.0 / dt)), f"blowup-{N}")


@dataclass
class Request:
    """One serving request: an HBE solve submitted at `arrival` seconds."""
    rid: int
    arrival: float
    N: int
    L: float
    mu: float
    lam: float
    T: float
    bumps: List[Tuple[float, float, Tuple[float, float, float]]] = field(default_factory=list)

    def initial(self) -> Tuple[np.ndarray, np.ndarray]:
        phi0 = np.zeros((self.N, self.N, self.N))
        for A, R, c in self.bumps:
            bump_into(phi0, self.L, DIRICHLET, A, R, c)
        return phi0, np.zeros_like(phi0)

    def steps(self) -> Tuple[int, float]:
        return steps_for(self.T, grid_spacing(self.N, self.L, DIRICHLET))


SERVE_SIZES = (32, 48, 64, 96, 128, 192, 256)


def request_stream(count: int = 256, seed: int = 0, rate: float = 1.0,
                   sizes: Sequence[int] = SERVE_SIZES) -> List[Request]:
    """Seeded Poisson stream of solve requests: box [-10, 10]^3 (L = 20),
    zero-Dirichlet, N uniform over `sizes`, mu, lambda ~ U[0.5, 2], 1-4 bumps with
    A ~ U[-2, 2], R ~ U[1, 4], centre ~ U[-4, 4]^3, phi1 = 0, horizon T ~ U[1, 6].
    Inter-arrival times are exponential with the given rate (requests / s)."""
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    for rid in range(count):
        t += rng.exponential(1.0 / rate)
        N = int(rng.choice(np.asarray(sizes)))
        mu = float(rng.uniform(0.5, 2.0))
        lam = float(rng.uniform(0.5, 2.0))
        nb = int(rng.integers(1, 5))
        bumps = []
        for _ in range(nb):
            A = float(rng.uniform(-2.0, 2.0))
            R = float(rng.uniform(1.0, 4.0))
            c = tuple(float(v) for v in rng.uniform(-4.0, 4.0, size=3))
            bumps.append((A, R, c))
        T = float(rng.uniform(1.0, 6.0))
        out.append(Request(rid, t, N, 20.0, mu, lam, T, bumps))
    return out
