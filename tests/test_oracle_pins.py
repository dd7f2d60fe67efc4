"""Pins of the CPU oracle against what the paper and the mathematics fix.

Each test checks the oracle (oracle/hbe_oracle.c, the plain FP64 RK4 + FD4
restatement of Sec. 2.1) against something other than itself: a library ODE
solver, a closed form, an invariant, a second discretisation, or brute force.
Together they are chosen so that a dropped term, a wrong sign, a wrong index or
a wrong RK4 weight fails at least one of them.
"""
import math

import numpy as np
import pytest
from scipy import ndimage
from scipy.integrate import solve_ivp
from scipy.interpolate import CubicSpline
from scipy.special import jv, yv

import hbe_inputs as hi
import oracle
from oracle import radial
from oracle import radial_phi

D, P = oracle.DIRICHLET, oracle.PERIODIC


def duffing_ode(mu, lam, a0, b0, T, rtol=1e-13):
    """phi'' + 3 phi' = mu^2 phi - lambda phi^3 (Eq. (duffing)) by DOP853."""
    sol = solve_ivp(lambda t, y: [y[1], -3.0 * y[1] + mu * mu * y[0] - lam * y[0] ** 3],
                    (0.0, T), [a0, b0], method="DOP853", rtol=rtol, atol=1e-15)
    return sol.y[0, -1], sol.y[1, -1]


# ---------------------------------------------------------------- P1 Duffing
def test_homogeneous_data_follows_duffing_ode():
    """Spatially constant data on the periodic grid: FD4 of a constant is zero
    (-1/6 + 8/3 - 5/2 = 0), so every node must follow the damped Duffing ODE."""
    N, L, mu, lam = 8, 4.0, 1.3, 0.7
    a0, b0 = 0.4, -0.2
    dt, n = 1e-3, 1000
    phi, psi, steps = oracle.run(np.full((N, N, N), a0), np.full((N, N, N), b0), L, mu, lam, P,
                                 0.0, dt, n)
    assert steps == n
    ya, yb = duffing_ode(mu, lam, a0, b0, n * dt)
    assert np.ptp(phi) == 0.0 and np.ptp(psi) == 0.0
    assert abs(phi[0, 0, 0] - ya) <= 1e-12
    assert abs(psi[0, 0, 0] - yb) <= 1e-12


def test_homogeneous_rk4_is_fourth_order_in_dt():
    """A wrong RK4 weight or stage time drops the order: the error against the
    ODE must shrink ~16x when dt halves."""
    N, L, mu, lam, T = 4, 4.0, 1.0, 1.0, 2.0
    ya, _ = duffing_ode(mu, lam, 1.5, 0.3, T)
    errs = []
    for n in (20, 40, 80):
        phi, _, _ = oracle.run(np.full((N, N, N), 1.5), np.full((N, N, N), 0.3), L, mu, lam, P,
                               0.0, T / n, n)
        errs.append(abs(phi[0, 0, 0] - ya))
    for e1, e2 in zip(errs, errs[1:]):
        assert 3.7 <= math.log2(e1 / e2) <= 4.3


def test_long_time_limit_is_paper_vacuum(paper_values):
    """Example 'long-bubble' (mu^2 = 9, lambda = 2) and the last example
    (mu^2 = lambda = 0.1): the Duffing limit values the paper prints."""
    N = 4
    phi, _, _ = oracle.run(np.full((N, N, N), 0.3), np.zeros((N, N, N)), 4.0, 3.0, 2.0, P,
                           0.0, 0.01, 2000)
    assert round(phi[0, 0, 0], 2) == paper_values["duffing_mu2_9_lambda_2"]
    phi, _, _ = oracle.run(np.full((N, N, N), -0.3), np.zeros((N, N, N)), 4.0, math.sqrt(0.1),
                           0.1, P, 0.0, 0.05, 4000)
    assert round(phi[0, 0, 0], 2) == -paper_values["duffing_mu2_0.1_lambda_0.1"]


def test_homogeneous_blowup_time_and_stop_rule():
    """Focusing case (lambda = -1) from 3/e at rest: the ODE passes 1e6 at
    t* ~ 1.939; the oracle stops after the first step past the threshold."""
    mu, lam, a0 = 1.0, -1.0, 3.0 / math.e
    ev = lambda t, y: abs(y[0]) - 1e6
    ev.terminal = True
    sol = solve_ivp(lambda t, y: [y[1], -3 * y[1] + mu * mu * y[0] - lam * y[0] ** 3], (0, 10),
                    [a0, 0.0], method="DOP853", rtol=1e-12, atol=1e-12, events=ev)
    t_star = sol.t_events[0][0]
    assert abs(t_star - 1.939) < 5e-3
    N, dt = 4, 1e-3
    phi, _, steps = oracle.run(np.full((N, N, N), a0), np.zeros((N, N, N)), 4.0, mu, lam, P, 0.0,
                               dt, 100000, stop_threshold=1e6)
    assert abs(phi[0, 0, 0]) > 1e6
    assert abs(steps * dt - t_star) <= 2 * dt
    # one step earlier the threshold was not yet crossed
    phi_prev, _, _ = oracle.run(np.full((N, N, N), a0), np.zeros((N, N, N)), 4.0, mu, lam, P,
                                0.0, dt, steps - 1)
    assert abs(phi_prev[0, 0, 0]) <= 1e6


# ---------------------------------------------------------------- P2 vacua
@pytest.mark.parametrize("sign", [1.0, -1.0])
def test_vacua_are_stationary(sign):
    N, mu, lam = 8, 1.7, 0.9
    v = sign * mu / math.sqrt(lam)
    phi, psi, _ = oracle.run(np.full((N, N, N), v), np.zeros((N, N, N)), 5.0, mu, lam, P, 0.0,
                             0.05, 200)
    assert np.max(np.abs(phi - v)) <= 8 * np.spacing(abs(v))
    assert np.max(np.abs(psi)) <= 1e-14


def test_zero_data_stays_zero_bitwise():
    N = 12
    for bc in (D, P):
        phi, psi, _ = oracle.run(np.zeros((N, N, N)), np.zeros((N, N, N)), 6.0, 1.0, 1.0, bc, 0.0,
                                 0.1, 30)
        assert not phi.any() and not psi.any()


# ---------------------------------------------------------------- P3 plane wave
def test_plane_wave_reduces_to_two_by_two_rk4():
    """lambda = 0: the grid solution is a(t) cos(k.x) exactly, where (a, a') obeys
    RK4 on a'' + 3a' + (e^{-2t} sigma_h - mu^2) a = 0, sigma_h the FD4 symbol
    summed over the axes; the recursion is run here in 40-digit arithmetic."""
    import mpmath as mp
    mp.mp.dps = 40
    N, L, mu = 16, 8.0, 1.1
    m = (1, 2, 1)
    h = L / N
    dt, n = h / 4, 12
    phi0 = hi.plane_wave(N, L, m)
    phi, psi, _ = oracle.run(phi0, np.zeros_like(phi0), L, mu, 0.0, P, 0.0, dt, n)
    sig = mp.mpf(0)
    for mi in m:
        k = 2 * mp.pi * mi / L
        sig += (mp.mpf(5) / 2 - mp.mpf(8) / 3 * mp.cos(k * h) + mp.mpf(1) / 6 * mp.cos(2 * k * h)) / mp.mpf(h) ** 2
    mu2, DT = mp.mpf(mu) ** 2, mp.mpf(dt)

    def f(t, a, b):
        return b, -3 * b - (mp.exp(-2 * t) * sig - mu2) * a

    a, b = mp.mpf(1), mp.mpf(0)
    for j in range(n):
        t = j * DT
        k1 = f(t, a, b)
        k2 = f(t + DT / 2, a + DT / 2 * k1[0], b + DT / 2 * k1[1])
        k3 = f(t + DT / 2, a + DT / 2 * k2[0], b + DT / 2 * k2[1])
        k4 = f(t + DT, a + DT * k3[0], b + DT * k3[1])
        a += DT / 6 * (k1[0] + 2 * k2[0] + 2 * k3[0] + k4[0])
        b += DT / 6 * (k1[1] + 2 * k2[1] + 2 * k3[1] + k4[1])
    assert np.max(np.abs(phi - float(a) * phi0)) <= 1e-13
    assert np.max(np.abs(psi - float(b) * phi0)) <= 1e-13


def _bessel_amplitude(k, mu, T):
    """Continuum a(T) for a'' + 3a' + (e^{-2t}k^2 - mu^2) a = 0, a(0) = 1, a'(0) = 0:
    a = e^{-3t/2} [c1 J_M(k e^{-t}) + c2 Y_M(k e^{-t})], M = sqrt(mu^2 + 9/4)."""
    M = math.sqrt(mu * mu + 9.0 / 4.0)

    def basis(t):
        s = k * math.exp(-t)
        return np.array([math.exp(-1.5 * t) * jv(M, s), math.exp(-1.5 * t) * yv(M, s)])

    def dbasis(t):
        # d/dt [e^{-3t/2} Z_M(k e^{-t})] = e^{-3t/2} [-3/2 Z_M(s) - s Z_M'(s)], Z' = (Z_{M-1} - Z_{M+1}) / 2
        s = k * math.exp(-t)
        e = math.exp(-1.5 * t)
        dj = 0.5 * (jv(M - 1, s) - jv(M + 1, s))
        dy = 0.5 * (yv(M - 1, s) - yv(M + 1, s))
        return np.array([e * (-1.5 * jv(M, s) - s * dj), e * (-1.5 * yv(M, s) - s * dy)])

    c = np.linalg.solve(np.array([basis(0.0), dbasis(0.0)]), [1.0, 0.0])
    return float(c @ basis(T))


def test_plane_wave_converges_to_bessel_closed_form():
    """lambda = 0 plane wave against the closed form of the transformed equation
    (Eq. (K_G_Higgs) with u = e^{3t/2} phi is Bessel's equation in k e^{-t}):
    error O(h^4) at dt = h/4."""
    L, mu, T = 8.0, 1.0, 1.0
    m = (1, 0, 0)
    k = 2 * math.pi / L
    aT = _bessel_amplitude(k, mu, T)
    errs = []
    for N in (8, 16, 32):
        h = L / N
        n = int(round(T / (h / 4)))
        phi0 = hi.plane_wave(N, L, m)
        phi, _, _ = oracle.run(phi0, np.zeros_like(phi0), L, mu, 0.0, P, 0.0, T / n, n)
        mask = np.abs(phi0) > 0.5
        errs.append(np.max(np.abs(phi[mask] / phi0[mask] - aT)))
    assert errs[-1] < 2e-6
    for e1, e2 in zip(errs, errs[1:]):
        assert 3.6 <= math.log2(e1 / e2) <= 4.4


# ---------------------------------------------------------------- P4 radial
def test_radial_data_matches_radial_solver():
    """Radially symmetric bump (1.5 exp(-1/(1 - r^2/9)) on [-5, 5]^3, mu = lambda = 1)
    against a fine-grid 1D solver in u = r phi (Sec. 2.2 equivalence); the
    discrepancy must shrink with h."""
    T = 1.0

    def f0(r):
        return np.where(r < 3, 1.5 * np.exp(-1.0 / np.maximum(1 - r * r / 9.0, 1e-300)), 0.0)

    R, Mr = 8.0, 4000
    r, ph = radial.solve(f0, lambda r: 0.0 * r, R, Mr, 1.0, 1.0, T, R / Mr / 4)
    ref = CubicSpline(r, ph)
    errs, cerr = [], []
    for N in (31, 63):
        prob = hi.radial_bump_problem(N)
        h = hi.grid_spacing(N, prob.L, D)
        n = int(round(T / (h / 4)))
        phi, _, _ = oracle.run(prob.phi0, prob.phi1, prob.L, prob.mu, prob.lam, D, 0.0, T / n, n)
        x = hi.grid_coords(N, prob.L, D)
        rr = np.sqrt(x[:, None, None] ** 2 + x[None, :, None] ** 2 + x[None, None, :] ** 2)
        m = rr < 4.5
        errs.append(np.max(np.abs(phi[m] - ref(rr[m]))))
        # the centre node sits at r = 0 for odd N
        cerr.append(abs(phi[N // 2, N // 2, N // 2] - ref(0.0)))
    assert errs[0] < 2e-3 and errs[1] < 5e-4
    assert errs[0] / errs[1] > 3.5
    assert cerr[0] < 1e-5 and cerr[1] < cerr[0] / 4


# ---------------------------------------------------------------- P5 symmetry
def test_octant_reflection_symmetry_is_bitwise():
    N, L = 24, 10.0
    x = hi.grid_coords(N, L, D)
    # even in each axis but not radial: different widths per axis
    phi0 = (1.2 * np.exp(-x[None, None, :] ** 2 / 2.0) * np.exp(-x[None, :, None] ** 2 / 3.0)
            * np.exp(-x[:, None, None] ** 2 / 1.5))
    phi1 = -0.5 * phi0
    phi, psi, _ = oracle.run(phi0, phi1, L, 1.2, 0.8, D, 0.0, 0.05, 20)
    for ax in range(3):
        assert np.array_equal(phi, np.flip(phi, axis=ax))
        assert np.array_equal(psi, np.flip(psi, axis=ax))


def test_axis_permutation_symmetry():
    prob = hi.radial_bump_problem(24)
    phi, _, _ = oracle.run(prob.phi0, prob.phi1, prob.L, prob.mu, prob.lam, D, 0.0, prob.dt, 20)
    s = np.max(np.abs(phi))
    for perm in [(1, 0, 2), (2, 1, 0), (0, 2, 1)]:
        assert np.max(np.abs(phi - np.transpose(phi, perm))) <= 1e-14 * s


# ---------------------------------------------------------------- P6 convergence
def test_observed_fourth_order_convergence():
    """Self-convergence on nested periodic grids (h, h/2, h/4) at dt = h/4 with
    smooth nonlinear data: log2 of successive difference ratios in [3.7, 4.3]."""
    L, T, mu, lam = 8.0, 1.0, 1.3, 1.0
    sols = {}
    for N in (32, 64, 128):
        x = hi.grid_coords(N, L, P)
        k = 2 * math.pi / L
        X, Y, Z = x[None, None, :], x[None, :, None], x[:, None, None]
        phi0 = (0.5 * np.cos(k * X) * np.cos(2 * k * Y) + 0.3 * np.sin(k * Z + 0.3)
                + 0.2 * np.cos(k * (X + Y + Z)))
        phi1 = 0.2 * np.sin(k * X) * np.cos(k * Z) + 0 * Y
        h = L / N
        n = int(round(T / (h / 4)))
        sols[N], _, _ = oracle.run(np.ascontiguousarray(phi0), np.ascontiguousarray(phi1), L, mu,
                                   lam, P, 0.0, T / n, n)
    e1 = np.max(np.abs(sols[32] - sols[64][::2, ::2, ::2]))
    e2 = np.max(np.abs(sols[64] - sols[128][::2, ::2, ::2]))
    assert 3.7 <= math.log2(e1 / e2) <= 4.3


# ---------------------------------------------------------------- P7 FD4
def test_fd4_exact_on_quintic_polynomials():
    N, h = 16, 0.37
    x = (np.arange(N) - 7.3) * h
    X, Y, Z = x[None, None, :], x[None, :, None], x[:, None, None]
    u = (X ** 5 - 2 * X ** 3 * Y ** 2 + 3 * Y ** 4 * Z - Z ** 5 + X * Y * Z ** 3 + 2 * X ** 2 - 1)
    lap_exact = (20 * X ** 3 - 12 * X * Y ** 2 - 4 * X ** 3 + 36 * Y ** 2 * Z - 20 * Z ** 3
                 + 6 * X * Y * Z + 4)
    lap = oracle.laplacian(np.ascontiguousarray(u + 0 * X * Y * Z), h, D)
    inner = (slice(2, -2),) * 3  # away from the zero ghosts
    scale = np.max(np.abs(u))
    assert np.max(np.abs(lap[inner] - lap_exact[inner])) <= 1e-10 * scale / (h * h)


def test_fd4_error_term_on_sextic():
    """FD4 of x^6 is exactly 30 x^4 - 8 h^4 (leading error -(h^4/90) f^(6))."""
    N, h = 12, 0.5
    x = (np.arange(N) - 5.0) * h
    u = np.broadcast_to(x[None, None, :] ** 6, (N, N, N)).copy()
    lap = oracle.laplacian(u, h, D)
    xi = x[2:-2]
    assert np.allclose(lap[5, 5, 2:-2], 30 * xi ** 4 - 8 * h ** 4, rtol=0, atol=1e-9)


def test_fd4_weights_are_the_papers(paper_values):
    """The Laplacian of a unit spike returns the printed weights (Sec. 2.1),
    including the merged 3D centre coefficient -15/2."""
    N, h = 9, 1.0
    u = np.zeros((N, N, N))
    u[4, 4, 4] = 1.0
    lap = oracle.laplacian(u, h, D)
    assert lap[4, 4, 4] == paper_values["fd4_centre_3d"]
    for off, key in ((1, "fd4_w1"), (2, "fd4_w2")):
        for sl in ((4, 4, 4 + off), (4, 4, 4 - off), (4, 4 + off, 4), (4, 4 - off, 4),
                   (4 + off, 4, 4), (4 - off, 4, 4)):
            assert abs(lap[sl] - paper_values[key]) < 1e-15
    assert np.count_nonzero(lap) == 13


# ---------------------------------------------------------------- P12 zero-Dirichlet wall
# Eq. (BC) with the 5-wide stencil of Sec. 2.1 needs two ghost layers; the
# reading taken (C3) is that both hold 0 for every field.  The 1D operator is
# then the banded N x N matrix of the FD4 weights with the rows simply cut off
# at the matrix edge, and the 3D operator is its Kronecker sum over the axes.
# Neither is built from the oracle's own node() rule.
def _fd4_truncated_matrix(N, h):
    w = (-1.0 / 12.0, 4.0 / 3.0, -5.0 / 2.0, 4.0 / 3.0, -1.0 / 12.0)
    D1 = np.zeros((N, N))
    for i in range(N):
        for o in range(-2, 3):
            if 0 <= i + o < N:
                D1[i, i + o] = w[o + 2] / (h * h)
    return D1


def _kron_laplacian(u, h):
    """(D x I x I + I x D x I + I x I x D) u for u indexed [z, y, x]."""
    from scipy import sparse
    N = u.shape[0]
    D1 = sparse.csr_matrix(_fd4_truncated_matrix(N, h))
    I = sparse.identity(N, format="csr")
    A = (sparse.kron(sparse.kron(I, I), D1) + sparse.kron(sparse.kron(I, D1), I)
         + sparse.kron(sparse.kron(D1, I), I))
    return (A @ u.ravel()).reshape(u.shape)


def _wall_mismatch(lap):
    """Largest relative disagreement of `lap(u, h)` with the truncated banded
    operator: on a random field (all nodes, reported separately for the two
    layers next to each wall) and on unit spikes at the corner nodes."""
    N, h = 11, 0.37
    rng = np.random.default_rng(12)
    u = rng.standard_normal((N, N, N))
    got, want = lap(u, h), _kron_laplacian(u, h)
    scale = np.max(np.abs(want))
    err = np.max(np.abs(got - want)) / scale
    wall = [0, 1, N - 2, N - 1]
    for ax in range(3):
        sl = [slice(None)] * 3
        sl[ax] = wall
        err = max(err, np.max(np.abs(got[tuple(sl)] - want[tuple(sl)])) / scale)
    # a unit spike on a corner returns the truncated weights: the centre sums
    # three -5/2 terms, each axis keeps only its inward +1 and +2 neighbours
    for c in (0, N - 1):
        e = np.zeros((N, N, N))
        e[c, c, c] = 1.0
        g = lap(e, 1.0)
        s = 1 if c == 0 else -1
        want_s = np.zeros((N, N, N))
        want_s[c, c, c] = -7.5
        for ax in range(3):
            for o, wgt in ((1, 4.0 / 3.0), (2, -1.0 / 12.0)):
                idx = [c, c, c]
                idx[ax] = c + s * o
                want_s[tuple(idx)] = wgt
        err = max(err, np.max(np.abs(g - want_s)) / 7.5)
    return err


def test_dirichlet_wall_is_truncated_banded_operator():
    """The oracle's FD4 Laplacian at and next to the zero-Dirichlet wall equals
    the banded matrix truncated at the two zero ghost layers (reading C3 of
    Eq. BC) to rounding."""
    assert _wall_mismatch(lambda u, h: oracle.laplacian(u, h, D)) <= 1e-13


_WALL_RULE = ("  if (i < 0 || i >= g->nx || j < 0 || j >= g->ny || k < 0 || k >= g->nz) "
              "return 0.0;")
_WALL_MUTANTS = {
    # odd reflection about the wall node (index -1): u(-2) = -u(0)
    "odd_reflection": (
        "  if (i == -2) return -node(u, g, 0, j, k);\n"
        "  if (i == g->nx + 1) return -node(u, g, g->nx - 1, j, k);\n"
        "  if (j == -2) return -node(u, g, i, 0, k);\n"
        "  if (j == g->ny + 1) return -node(u, g, i, g->ny - 1, k);\n"
        "  if (k == -2) return -node(u, g, i, j, 0);\n"
        "  if (k == g->nz + 1) return -node(u, g, i, j, g->nz - 1);\n" + _WALL_RULE),
    # a single zero ghost layer; the second one mirrors the first interior node
    "one_ghost_layer": (
        "  if (i == -2) i = 0;\n  if (i == g->nx + 1) i = g->nx - 1;\n"
        "  if (j == -2) j = 0;\n  if (j == g->ny + 1) j = g->ny - 1;\n"
        "  if (k == -2) k = 0;\n  if (k == g->nz + 1) k = g->nz - 1;\n" + _WALL_RULE),
    # off-by-one bounds: the last interior node read as a ghost
    "off_by_one_upper": _WALL_RULE.replace("i >= g->nx", "i >= g->nx - 1")
                                  .replace("j >= g->ny", "j >= g->ny - 1")
                                  .replace("k >= g->nz", "k >= g->nz - 1"),
    # off-by-one bounds: the first interior node read as a ghost
    "off_by_one_lower": _WALL_RULE.replace("i < 0", "i < 1").replace("j < 0", "j < 1")
                                  .replace("k < 0", "k < 1"),
}


@pytest.mark.parametrize("mutant", sorted(_WALL_MUTANTS))
def test_dirichlet_wall_pin_rejects_planted_mistakes(mutant, tmp_path):
    """Plant a plausible wall mistake in a copy of the oracle's C source, build
    it, and check that the wall pin above rejects it."""
    import ctypes
    import subprocess
    src = open(oracle._SRC).read()
    assert src.count(_WALL_RULE) == 1
    path = tmp_path / "mut.c"
    path.write_text(src.replace(_WALL_RULE, _WALL_MUTANTS[mutant]))
    so = tmp_path / "libmut.so"
    subprocess.run(["gcc", "-O1", "-std=c11", "-ffp-contract=off", "-shared", "-fPIC", "-o",
                    str(so), str(path), "-lm"], check=True)
    lib = ctypes.CDLL(str(so))
    dp = ctypes.POINTER(ctypes.c_double)
    lib.oracle_laplacian.argtypes = [dp, dp, ctypes.c_int, ctypes.c_double, ctypes.c_int,
                                     ctypes.c_int]
    lib.oracle_laplacian.restype = None

    def lap(u, h):
        u = np.ascontiguousarray(u, dtype=np.float64)
        out = np.empty_like(u)
        lib.oracle_laplacian(u.ctypes.data_as(dp), out.ctypes.data_as(dp), u.shape[0], h, D, 1)
        return out

    assert _wall_mismatch(lap) > 1e-3


def test_even_closure_at_origin(paper_values):
    """For data even about a node the FD4 x-derivative there collapses to the
    paper's origin closure (-5/2, 8/3, -1/6) / dr^2 (Sec. 2.2)."""
    N, h = 9, 0.25
    rng = np.random.default_rng(3)
    half = rng.standard_normal(5)
    row = np.concatenate([half[:0:-1], half])  # even about index 4
    u = np.broadcast_to(row[None, None, :], (N, N, N)).copy()
    lap = oracle.laplacian(u, h, D)
    w0, w1, w2 = paper_values["radial_origin"]
    want = (w0 * half[0] + w1 * half[1] + w2 * half[2]) / h ** 2
    # y and z second differences of a y,z-constant field vanish away from the walls
    assert abs(lap[4, 4, 4] - want) <= 1e-12 * max(1.0, abs(want))


# ---------------------------------------------------------------- P8 RK4 polynomial
@pytest.mark.parametrize("mu,dt", [(1.0, 0.1), (2.0, 0.05)])
def test_rk4_amplification_on_linear_modes(mu, dt):
    """lambda = 0, constant data: the system matrix [[0, 1], [mu^2, -3]] has
    eigenvalues r = -3/2 +- M; starting on an eigenvector one RK4 step multiplies
    by R(z) = 1 + z + z^2/2 + z^3/6 + z^4/24, z = r dt."""
    M = math.sqrt(mu * mu + 9.0 / 4.0)
    N = 4
    for r in (-1.5 + M, -1.5 - M):
        phi, psi, _ = oracle.run(np.full((N, N, N), 1.0), np.full((N, N, N), r), 4.0, mu, 0.0, P,
                                 0.0, dt, 1)
        z = r * dt
        R = 1 + z + z * z / 2 + z ** 3 / 6 + z ** 4 / 24
        assert abs(phi[0, 0, 0] - R) <= 1e-15 * 4
        assert abs(psi[0, 0, 0] - R * r) <= 1e-15 * 4 * abs(r) + 1e-16


# ---------------------------------------------------------------- P9 linearity / shift
def test_superposition_for_lambda_zero():
    N, L = 16, 8.0
    rng = np.random.default_rng(7)
    a0, a1, b0, b1 = (rng.standard_normal((N, N, N)) for _ in range(4))
    args = (L, 1.1, 0.0, D, 0.0, 0.05, 10)
    pa, qa, _ = oracle.run(a0, a1, *args)
    pb, qb, _ = oracle.run(b0, b1, *args)
    pc, qc, _ = oracle.run(a0 + b0, a1 + b1, *args)
    s = max(np.max(np.abs(pa)), np.max(np.abs(pb)))
    assert np.max(np.abs(pc - pa - pb)) <= 1e-12 * s
    # the nonlinear term breaks superposition: lambda != 0 must not pass
    pa, _, _ = oracle.run(a0, a1, L, 1.1, 1.0, D, 0.0, 0.05, 10)
    pb, _, _ = oracle.run(b0, b1, L, 1.1, 1.0, D, 0.0, 0.05, 10)
    pc, _, _ = oracle.run(a0 + b0, a1 + b1, L, 1.1, 1.0, D, 0.0, 0.05, 10)
    assert np.max(np.abs(pc - pa - pb)) > 1e-3


def test_periodic_shift_is_bitwise():
    N, L = 16, 8.0
    rng = np.random.default_rng(11)
    a0, a1 = rng.standard_normal((N, N, N)), rng.standard_normal((N, N, N))
    pa, qa, _ = oracle.run(a0, a1, L, 1.0, 1.0, P, 0.0, 0.05, 5)
    sh = (3, -5, 7)
    pb, qb, _ = oracle.run(np.roll(a0, sh, axis=(0, 1, 2)), np.roll(a1, sh, axis=(0, 1, 2)), L, 1.0,
                           1.0, P, 0.0, 0.05, 5)
    assert np.array_equal(pb, np.roll(pa, sh, axis=(0, 1, 2)))
    assert np.array_equal(qb, np.roll(qa, sh, axis=(0, 1, 2)))


# ---------------------------------------------------------------- time origin
def test_time_origin_enters_through_e_minus_2t():
    """Starting at t0 = s with the box side scaled by e^{-s} is the same
    problem (e^{-2t} Delta is invariant under t -> t + s, x -> e^{-s} x)."""
    N = 16
    rng = np.random.default_rng(5)
    a0 = rng.standard_normal((N, N, N))
    s = 0.7
    p1, _, _ = oracle.run(a0, 0 * a0, 8.0, 1.0, 1.0, P, 0.0, 0.01, 20)
    p2, _, _ = oracle.run(a0, 0 * a0, 8.0 * math.exp(-s), 1.0, 1.0, P, s, 0.01, 20)
    assert np.max(np.abs(p1 - p2)) <= 1e-12 * np.max(np.abs(p1))


# ---------------------------------------------------------------- diagnostics
def _components_library(mask, periodic):
    """Connected components (6-connectivity) by scipy.ndimage.label; periodic
    wrap by merging labels that touch across opposite faces."""
    lab, n = ndimage.label(mask, structure=ndimage.generate_binary_structure(3, 1))
    if not periodic or n == 0:
        return n
    parent = list(range(n + 1))

    def find(a):
        while parent[a] != a:
            parent[a] = parent[parent[a]]
            a = parent[a]
        return a

    for ax in range(3):
        a = np.take(lab, 0, axis=ax)
        b = np.take(lab, -1, axis=ax)
        for u, v in zip(a.ravel(), b.ravel()):
            if u and v:
                ru, rv = find(u), find(v)
                if ru != rv:
                    parent[ru] = rv
    return len({find(i) for i in range(1, n + 1)})


@pytest.mark.parametrize("bc", [D, P])
@pytest.mark.parametrize("seed", [0, 1, 2])
def test_sign_components_match_library_labelling(bc, seed):
    N = 20
    rng = np.random.default_rng(seed)
    phi = ndimage.gaussian_filter(rng.standard_normal((N, N, N)), 1.5,
                                  mode="wrap" if bc == P else "constant")
    phi[rng.random((N, N, N)) < 0.02] = 0.0  # exact zeros belong to neither sign
    d = oracle.diag(phi, bc)
    assert d["n_pos"] == _components_library(phi > 0, bc == P)
    assert d["n_neg"] == _components_library(phi < 0, bc == P)
    assert d["bubble_count"] == max(0, d["n_pos"] + d["n_neg"] - 1)
    assert d["max_abs_phi"] == np.max(np.abs(phi)) and d["finite"]
    # masks: bit x % 32 of word x // 32 of row (z, y)
    W = (N + 31) // 32
    bits = np.unpackbits(d["pos_mask"].view(np.uint8), bitorder="little").reshape(N, N, W * 32)
    assert np.array_equal(bits[:, :, :N].astype(bool), phi > 0)
    bits = np.unpackbits(d["neg_mask"].view(np.uint8), bitorder="little").reshape(N, N, W * 32)
    assert np.array_equal(bits[:, :, :N].astype(bool), phi < 0)


def test_bubble_count_on_constructed_fields():
    N, L = 32, 10.0
    x = hi.grid_coords(N, L, D)
    r = np.sqrt(x[None, None, :] ** 2 + x[None, :, None] ** 2 + x[:, None, None] ** 2)
    # negative core inside a positive shell inside exact zeros: one bubble
    phi = np.where(r < 2, -1.0, np.where(r < 4, 1.0, 0.0))
    d = oracle.diag(phi, D)
    assert (d["n_pos"], d["n_neg"], d["bubble_count"]) == (1, 1, 1)
    # two separated negative balls in a positive sea: two bubbles
    xx = x[None, None, :]
    phi = np.ones((N, N, N))
    phi[np.sqrt((xx - 2.5) ** 2 + x[None, :, None] ** 2 + x[:, None, None] ** 2) < 1.5] = -1.0
    phi[np.sqrt((xx + 2.5) ** 2 + x[None, :, None] ** 2 + x[:, None, None] ** 2) < 1.5] = -1.0
    d = oracle.diag(phi, D)
    assert (d["n_pos"], d["n_neg"], d["bubble_count"]) == (1, 2, 2)
    # one sign only: no bubble
    d = oracle.diag(np.abs(phi), D)
    assert d["bubble_count"] == 0
    # periodic wrap joins slabs touching the opposite faces
    phi = -np.ones((N, N, N))
    phi[:, :, :3] = 1.0
    phi[:, :, -3:] = 1.0
    assert oracle.diag(phi, P)["n_pos"] == 1
    assert oracle.diag(phi, D)["n_pos"] == 2


def test_nonfinite_is_flagged():
    phi = np.zeros((8, 8, 8))
    phi[1, 2, 3] = np.nan
    assert not oracle.diag(phi, D)["finite"]
    phi[1, 2, 3] = np.inf
    assert not oracle.diag(phi, D)["finite"]


# ---------------------------------------------------------------- one-point windows
@pytest.mark.parametrize("bc", [D, P])
def test_window_values_equal_full_grid_values(bc):
    """The one-point window evaluation used for full-size parity samples is the
    full-grid oracle at those points, bit for bit (edge and interior points)."""
    N, L, nsteps = 40, 12.0, 2
    rng = np.random.default_rng(4)
    phi0 = ndimage.gaussian_filter(rng.standard_normal((N, N, N)), 2.0,
                                   mode="wrap" if bc == P else "constant")
    phi1 = 0.3 * np.roll(phi0, 3, axis=1)
    dt = hi.grid_spacing(N, L, bc) / 4
    pf, qf, _ = oracle.run(phi0, phi1, L, 1.0, 1.0, bc, 0.3, dt, nsteps)
    pts = [(0, 0, 0), (39, 20, 1), (20, 20, 20), (5, 38, 39), (17, 0, 33)]
    w = oracle.window_values(phi0, phi1, L, 1.0, 1.0, bc, 0.3, dt, nsteps, pts)
    for i, pt in enumerate(pts):
        assert w[i, 0] == pf[pt] and w[i, 1] == qf[pt]


# ---------------------------------------------------------------- P11 radial phi form (Sec. 2.2)
def test_radial_phi_operator_exact_on_even_polynomials():
    """phi_rr + (2/r) phi_r of r^2 is 6 and of r^4 is 20 r^2, at the origin
    too (3 phi_rr(0) with the even closure); FD4 and the even ghosts are exact
    on these, so only rounding remains away from the two wall nodes."""
    n, R = 40, 4.0
    dr = R / n
    r = np.arange(n) * dr
    inner = slice(0, n - 2)
    l2 = radial_phi.laplacian(r ** 2, dr)
    l4 = radial_phi.laplacian(r ** 4, dr)
    assert np.max(np.abs(l2[inner] - 6.0)) < 1e-10
    assert np.max(np.abs(l4[inner] - 20.0 * r[inner] ** 2)) < 1e-9
    assert abs(l2[0] - 6.0) < 1e-12 and abs(l4[0]) < 1e-12


def test_radial_phi_spherical_mode_matches_ode_at_fourth_order():
    """lambda = 0: phi = a(t) sin(kr)/(kr) with k = 3 pi / R (zero at the wall)
    solves Eq. (radial) when a'' + 3a' + (e^{-2t} k^2 - mu^2) a = 0 (DOP853).
    Away from the wall (where the zero ghosts act) the grid error falls 16x per
    halving of dr."""
    R, mu, T = 10.0, 1.0, 1.0
    k = 3 * math.pi / R
    sol = solve_ivp(lambda t, y: [y[1], -3 * y[1] - (math.exp(-2 * t) * k * k - mu * mu) * y[0]],
                    (0, T), [1.0, 0.0], method="DOP853", rtol=1e-13, atol=1e-15)
    a = sol.y[0, -1]
    errs = []
    for n in (100, 200, 400):
        dr = R / n
        r = np.arange(n) * dr
        phi0 = np.sinc(k * r / math.pi)
        nst = int(round(T / (dr / 4)))
        out = radial_phi.run(phi0, 0 * phi0, R, mu, 0.0, 0.0, T / nst, nst)
        sel = r <= R - 2
        errs.append(np.max(np.abs(out["phi"][sel] - a * phi0[sel])))
    assert errs[-1] < 1e-9
    for e1, e2 in zip(errs, errs[1:]):
        assert 3.8 <= math.log2(e1 / e2) <= 4.2


def test_radial_phi_agrees_with_u_form_solver():
    """The paper's phi form and the u = r phi form are different
    discretisations of the same problem: on a bump (mu = lambda = 1, t = 1)
    they agree to O(dr^4), including the origin value."""
    def f0(r):
        return np.where(r < 3, 1.5 * np.exp(-1.0 / np.maximum(1 - r * r / 9.0, 1e-300)), 0.0)

    ru, pu = radial.solve(f0, lambda r: 0 * r, 8.0, 4000, 1.0, 1.0, 1.0, 8.0 / 4000 / 4)
    ref = CubicSpline(ru, pu)
    errs = []
    for n in (200, 400):
        dr = 8.0 / n
        r = np.arange(n) * dr
        nst = int(round(1.0 / (dr / 4)))
        out = radial_phi.run(f0(r), 0 * r, 8.0, 1.0, 1.0, 0.0, 1.0 / nst, nst)
        sel = (r > 0) & (r < 6)
        errs.append(np.max(np.abs(out["phi"][sel] - ref(r[sel]))))
        assert abs(out["phi"][0] - ref(0.0)) < 1e-8
    assert errs[1] < 1e-6 and errs[0] / errs[1] > 10


def test_radial_phi_sign_changes_and_stop_rule():
    assert radial_phi.sign_changes(np.array([1.0, 0.5, -0.2, 0.0, -1e-9, 0.3]), 1e-6) == 2
    assert radial_phi.sign_changes(np.array([0.0, 0.0]), 0.0) == 0
    assert radial_phi.sign_changes(np.array([-1.0, -2.0, 3.0]), 0.0) == 1
    # focusing data: the run ends after the first step above the threshold
    n, R = 100, 10.0
    r = np.arange(n) * R / n
    phi0 = 3.0 * np.exp(-r * r)
    out = radial_phi.run(phi0, 0 * r, R, 1.0, -1.0, 0.0, 0.025, 400, stop=1e3)
    assert out["status"] == 1 and out["steps"] < 400
    assert np.max(np.abs(out["phi"])) > 1e3
    prev = radial_phi.run(phi0, 0 * r, R, 1.0, -1.0, 0.0, 0.025, out["steps"] - 1)
    assert np.max(np.abs(prev["phi"])) <= 1e3


# ---------------------------------------------------------------- input generators
def test_grid_is_symmetric_and_spacing_matches_rule():
    for N in (7, 8, 64):
        x = hi.grid_coords(N, 10.0, D)
        assert np.array_equal(x, -x[::-1])
        assert hi.grid_spacing(N, 10.0, D) == oracle.grid_spacing(N, 10.0, D)
        assert abs((x[0] + 5.0) - hi.grid_spacing(N, 10.0, D)) < 1e-14
    xp = hi.grid_coords(8, 8.0, P)
    assert xp[0] == -4.0 and xp[4] == 0.0


def test_grf_statistics():
    f = hi.grf(32, 40.0, seed=0)
    assert abs(f.mean()) < 1e-12 and abs(f.std() - 1.0) < 1e-12
    assert np.array_equal(f, hi.grf(32, 40.0, seed=0))
    assert not np.array_equal(f, hi.grf(32, 40.0, seed=1))
