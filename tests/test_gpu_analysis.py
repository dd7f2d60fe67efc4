"""The Sec. 3 analysis quantities computed on the device (hbe_analysis) against
their definitions evaluated on the same field on the host: h^3 sum phi,
h^3 sum phi^3, e^{-2t} max |FD4 Laplacian| (the oracle's Laplacian), and the
first bubble condition of the corollary quoted in Example 3."""
import math

import numpy as np
import pytest

import __graft_entry__  # noqa: F401
import hbe_inputs as hi
import oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hbe():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_1803_01291_gb300 as m
    return m


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("bc", [0, 1])
def test_analysis_matches_definitions(hbe, prec, bc):
    N, L, mu, lam = 36, 10.0, 3.0, 2.0
    rng = np.random.default_rng(bc)
    from scipy import ndimage
    mode = "wrap" if bc == 1 else "constant"
    phi0 = ndimage.gaussian_filter(rng.standard_normal((N, N, N)), 2.0, mode=mode) * 3
    phi1 = -5 * phi0 + 0.1 * ndimage.gaussian_filter(rng.standard_normal((N, N, N)), 2.0, mode=mode)
    h = hi.grid_spacing(N, L, bc)
    with hbe.Solver(N, L, mu, lam, bc, prec) as s:
        s.set_initial(phi0, phi1)
        s.step(5, h / 4)
        phi, psi, t = s.read()
        a = s.analysis(eps=1e-3)
    assert a["t"] == t
    assert math.isclose(a["integral_phi"], h ** 3 * math.fsum(phi.ravel()), rel_tol=1e-12, abs_tol=1e-12)
    assert math.isclose(a["integral_phi3"], h ** 3 * math.fsum((phi ** 3).ravel()), rel_tol=1e-12, abs_tol=1e-12)
    lap = oracle.laplacian(phi, h, bc)
    assert math.isclose(a["laplacian_monitor"], math.exp(-2 * t) * np.max(np.abs(lap)), rel_tol=1e-12)
    m = 1.5 + math.sqrt(2.25 + mu * mu)
    support = np.abs(phi) + np.abs(psi) > 1e-3
    assert a["support_points"] == int(support.sum())
    assert a["condition1_violations"] == int((support & (m * phi + psi >= 0)).sum())


def test_homogeneous_integral_is_volume_times_value(hbe):
    N, L = 16, 4.0
    with hbe.Solver(N, L, 1.0, 1.0, 1, 0) as s:
        s.set_initial(np.full((N, N, N), 0.7), np.zeros((N, N, N)))
        a = s.analysis()
    assert math.isclose(a["integral_phi"], 0.7 * L ** 3, rel_tol=1e-14)
    assert math.isclose(a["integral_phi3"], 0.7 ** 3 * L ** 3, rel_tol=1e-14)
    # the FD4 weights sum to zero; on a constant only rounding of the weighted
    # terms (a few ulp of 15/h^2 * 0.7) is left
    assert a["laplacian_monitor"] <= 1e-13


@pytest.mark.parametrize("prec", [1, 2])
def test_periodic_monitor_at_the_wrap(hbe, prec):
    """Periodic data whose largest Laplacian sits on the x = 0 face: after a few
    steps (compensated state with nonzero low parts) the monitor still equals
    its definition on the read field, so the wrap across the faces uses the
    current values."""
    N, L, mu, lam = 32, 10.0, 1.3, 0.7
    xs = hi.grid_coords(N, L, 1) + L / 2  # node 0 at 0: the x = 0 face
    k = 2 * math.pi / L
    # cos(k x) + 0.3 cos(2 k x): |phi_xx| peaks only at node 0, next to the wrap
    fx = np.cos(k * xs) + 0.3 * np.cos(2 * k * xs)
    phi0 = (fx[None, None, :] + 0.2 * np.sin(k * xs)[None, :, None]
            + 0.1 * np.cos(k * xs)[:, None, None]) * np.ones((N, N, N))
    phi1 = 0.3 * np.roll(phi0, 5, axis=2)
    h = hi.grid_spacing(N, L, 1)
    with hbe.Solver(N, L, mu, lam, 1, prec) as s:
        s.set_initial(phi0, phi1)
        s.step(7, h / 4)
        phi, psi, t = s.read()
        a = s.analysis()
    lap = oracle.laplacian(phi, h, 1)
    assert math.isclose(a["laplacian_monitor"], math.exp(-2 * t) * np.max(np.abs(lap)), rel_tol=1e-12)


@pytest.mark.parametrize("prec", [0, 1, 2, 3])
@pytest.mark.parametrize("bc", [0, 1])
def test_monitor_from_the_stage_pass(hbe, prec, bc):
    """P(t_n) recorded by the stages 1+2 kernel while stepping (11 steps: a full
    replay of 8 and one of 3) against e^{-2 t_n} max|Delta_h phi_n| of the
    oracle's Laplacian on the GPU's own state before each step, and stepping
    with the monitor on leaves the state bitwise unchanged."""
    N, L, mu, lam, n = 36, 10.0, 1.5, 1.0, 11
    rng = np.random.default_rng(40 + bc)
    from scipy import ndimage
    mode = "wrap" if bc == 1 else "constant"
    phi0 = ndimage.gaussian_filter(rng.standard_normal((N, N, N)), 2.0, mode=mode) * 3
    phi1 = ndimage.gaussian_filter(rng.standard_normal((N, N, N)), 2.0, mode=mode)
    h = hi.grid_spacing(N, L, bc)
    dt = h / 4
    # reference: the state before each step, stepped one at a time without the monitor
    want = []
    with hbe.Solver(N, L, mu, lam, bc, prec) as s:
        s.set_initial(phi0, phi1, 0.1)
        for i in range(n):
            phi, _, t = s.read(psi=False)
            lap = oracle.laplacian(phi, h, bc)
            want.append(math.exp(-2.0 * t) * np.max(np.abs(lap)))
            s.step(1, dt)
        ref_end = s.read(psi=False)[0]
    with hbe.Solver(N, L, mu, lam, bc, prec) as s:
        s.set_initial(phi0, phi1, 0.1)
        s.set_monitor(True)
        assert s.step(n, dt) == hbe.OK
        P, t = s.monitor(0, n)
        end = s.read(psi=False)[0]
        with pytest.raises(hbe.HBEError):
            s.monitor(0, n + 1)  # step n has not been taken
    assert np.array_equal(end, ref_end)
    assert np.allclose(t, 0.1 + np.arange(n) * dt, rtol=0, atol=1e-14)
    # FP64: the same Laplacian to rounding; FP32 family: the stencil of phi's
    # FP32 (high) part in FP32 arithmetic, against the full state in FP64
    tol = 1e-12 if prec == 0 else 2e-5
    assert np.max(np.abs(P - want) / np.array(want)) <= tol, (P, want)
