"""The allocation-free entry point hbe_step_fp64_noalloc, called through the C
ABI, against the allocating path (hbe_create + hbe_step, FP64) on the same
inputs, within the FP64 tolerance of the other GPU tests (1e-11 relative
max-norm), on two calls in a row with different sizes and boundaries (the
second call must not see anything the first left in the shared scratch).

It serves callers that cannot allocate device memory when they step: the test
allocates the input and output fields itself (as such a caller would, from
its own pool) and the library uses only its fixed device array.  This file is
named to be collected last."""
import ctypes

import numpy as np
import pytest

import __graft_entry__  # noqa: F401

pytestmark = pytest.mark.gpu

TOL = 1e-11


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_1803_01291_gb300 as hbe
    from paper_1803_01291_gb300 import _lib
    return torch, hbe, _lib.load()


def smooth(N, bc, seed):
    from scipy import ndimage
    rng = np.random.default_rng(seed)
    mode = "wrap" if bc == 1 else "constant"
    a = ndimage.gaussian_filter(rng.standard_normal((N, N, N)), 2.0, mode=mode) * 4
    b = ndimage.gaussian_filter(rng.standard_normal((N, N, N)), 2.0, mode=mode)
    return np.ascontiguousarray(a), np.ascontiguousarray(b)


def noalloc(torch, lib, N, L, mu, lam, bc, phi0, phi1, t0, dt, nsteps):
    a = torch.from_numpy(phi0).cuda()
    b = torch.from_numpy(phi1).cuda()
    out_phi = torch.full_like(a, float("nan"))
    out_psi = torch.full_like(a, float("nan"))
    stream = torch.cuda.current_stream().cuda_stream
    torch.cuda.synchronize()
    st = lib.hbe_step_fp64_noalloc(N, L, mu, lam, bc, ctypes.c_void_p(a.data_ptr()),
                                   ctypes.c_void_p(b.data_ptr()), t0, dt, nsteps,
                                   ctypes.c_void_p(out_phi.data_ptr()),
                                   ctypes.c_void_p(out_psi.data_ptr()), ctypes.c_void_p(stream))
    torch.cuda.synchronize()
    return st, out_phi.cpu().numpy(), out_psi.cpu().numpy()


def allocating(hbe, N, L, mu, lam, bc, phi0, phi1, t0, dt, nsteps):
    with hbe.Solver(N, L, mu, lam, bc, hbe.FP64) as s:
        s.set_initial(phi0, phi1, t0)
        s.step(nsteps, dt)
        phi, psi, _ = s.read()
    return phi, psi


def relerr(a, b):
    return np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300)


def test_noalloc_matches_allocating_path_on_two_calls(env):
    torch, hbe, lib = env
    cases = [  # (N, L, mu, lambda, bc, seed, t0, steps)
        (40, 12.0, 1.1, 0.9, 0, 3, 0.0, 6),
        (24, 8.0, 1.4, -0.5, 1, 4, 0.3, 5),
    ]
    for N, L, mu, lam, bc, seed, t0, nsteps in cases:
        phi0, phi1 = smooth(N, bc, seed)
        h = L / N if bc == 1 else L / (N + 1)
        dt = h / 4
        st, phi, psi = noalloc(torch, lib, N, L, mu, lam, bc, phi0, phi1, t0, dt, nsteps)
        assert st == 0, st
        ref_phi, ref_psi = allocating(hbe, N, L, mu, lam, bc, phi0, phi1, t0, dt, nsteps)
        assert np.all(np.isfinite(phi)) and np.all(np.isfinite(psi))
        assert relerr(phi, ref_phi) <= TOL
        assert relerr(psi, ref_psi) <= TOL


def test_noalloc_rejects_sizes_beyond_its_scratch(env):
    torch, hbe, lib = env
    N = 56
    phi0 = np.zeros((N, N, N))
    st, _, _ = noalloc(torch, lib, N, 10.0, 1.0, 1.0, 0, phi0, phi0, 0.0, 0.01, 1)
    assert st == 1  # HBE_EINVAL: the fixed scratch holds N <= 48


def test_noalloc_zero_steps_returns_the_initial_data(env):
    torch, hbe, lib = env
    N, bc = 20, 1
    phi0, phi1 = smooth(N, bc, 5)
    st, phi, psi = noalloc(torch, lib, N, 6.0, 1.0, 1.0, bc, phi0, phi1, 0.0, 0.05, 0)
    assert st == 0
    assert np.array_equal(phi, phi0) and np.array_equal(psi, phi1)


def test_noalloc_blowup_stops_like_the_allocating_path(env):
    """Focusing case (lambda < 0) from a large bump: the solve goes non-finite.
    Both paths return HBE_NONFINITE after the same step and hold the same
    state; one step fewer is a normal solve equal to the allocating one."""
    torch, hbe, lib = env
    N, L, mu, lam, bc = 24, 8.0, 1.0, -1.0, 0
    h = L / (N + 1)
    x = (np.arange(N) - (N - 1) / 2) * h
    r2 = x[None, None, :] ** 2 + x[None, :, None] ** 2 + x[:, None, None] ** 2
    phi0 = np.where(r2 < 9.0, 30.0 * np.exp(-1.0 / (1.0 - np.minimum(r2, 8.999) / 9.0)), 0.0)
    phi1 = np.zeros_like(phi0)
    dt, nsteps = h / 4, 40
    with hbe.Solver(N, L, mu, lam, bc, hbe.FP64) as s:
        s.set_initial(phi0, phi1)
        st_ref = s.step(nsteps, dt)
        n_stop, _ = s.progress()
        ref_phi, ref_psi, _ = s.read()
    assert st_ref == hbe.NONFINITE and 1 <= n_stop < nsteps
    st, phi, psi = noalloc(torch, lib, N, L, mu, lam, bc, phi0, phi1, 0.0, dt, nsteps)
    assert st == hbe.NONFINITE
    assert not np.all(np.isfinite(phi))
    same_state(phi, ref_phi)
    same_state(psi, ref_psi)
    # one step earlier phi is still finite (psi = phi_t may already have overflowed)
    st, phi, psi = noalloc(torch, lib, N, L, mu, lam, bc, phi0, phi1, 0.0, dt, n_stop - 1)
    assert st == 0
    ref_phi, ref_psi = allocating(hbe, N, L, mu, lam, bc, phi0, phi1, 0.0, dt, n_stop - 1)
    assert np.all(np.isfinite(phi))
    same_state(phi, ref_phi)
    same_state(psi, ref_psi)


def same_state(a, b):
    """Equal non-finite pattern (NaN, +-inf at the same nodes) and finite
    values within the FP64 tolerance."""
    fin = np.isfinite(b)
    assert np.array_equal(np.isfinite(a), fin)
    assert np.array_equal(np.isnan(a), np.isnan(b))
    assert np.array_equal(a[np.isinf(b)], b[np.isinf(b)])
    if fin.any():
        assert np.max(np.abs(a[fin] - b[fin])) <= TOL * max(np.max(np.abs(b[fin])), 1e-300)


def test_noalloc_rejects_a_non_finite_dt(env):
    torch, hbe, lib = env
    N = 16
    phi0 = np.zeros((N, N, N))
    st, _, _ = noalloc(torch, lib, N, 10.0, 1.0, 1.0, 0, phi0, phi0, 0.0, float("inf"), 1)
    assert st == 1
