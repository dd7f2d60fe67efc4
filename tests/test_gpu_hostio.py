"""Host input and output through the C ABI: page-locked host arrays are read
and written by the pack / unpack kernels directly, pageable arrays go through
device staging buffers.  Both routes must give the same bits, and the pinned
route must match the oracle like the others."""
import ctypes

import numpy as np
import pytest

import __graft_entry__  # noqa: F401
import hbe_inputs as hi
import oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_1803_01291_gb300 as m
    return torch, m


def rand_problem(N, bc, seed, L=12.0):
    from scipy import ndimage
    rng = np.random.default_rng(seed)
    mode = "wrap" if bc == 1 else "constant"
    phi0 = ndimage.gaussian_filter(rng.standard_normal((N, N, N)), 2.0, mode=mode) * 4
    phi1 = ndimage.gaussian_filter(rng.standard_normal((N, N, N)), 2.0, mode=mode)
    return phi0, phi1, L, hi.grid_spacing(N, L, bc) / 4


@pytest.mark.parametrize("bc", [0, 1])
@pytest.mark.parametrize("prec", [0, 1])
def test_pinned_and_pageable_host_buffers_agree(env, bc, prec):
    torch, hbe = env
    N, nsteps, mu, lam = 36, 4, 1.1, 0.9
    phi0, phi1, L, dt = rand_problem(N, bc, 7 + bc)
    dp = ctypes.POINTER(ctypes.c_double)
    out = {}
    for route in ("pageable", "pinned"):
        with hbe.Solver(N, L, mu, lam, bc, prec) as s:
            if route == "pinned":
                h0 = torch.from_numpy(phi0).pin_memory()
                h1 = torch.from_numpy(phi1).pin_memory()
                s.set_initial(h0.numpy(), h1.numpy())
            else:
                s.set_initial(phi0.copy(), phi1.copy())
            assert s.step(nsteps, dt) == hbe.OK
            if route == "pinned":
                pp = torch.full((N, N, N), float("nan"), dtype=torch.float64).pin_memory()
                pq = torch.full((N, N, N), float("nan"), dtype=torch.float64).pin_memory()
                t = ctypes.c_double()
                st = s.lib.hbe_read(s.handle, ctypes.cast(pp.data_ptr(), dp),
                                    ctypes.cast(pq.data_ptr(), dp), ctypes.byref(t))
                assert st == 0
                out[route] = (pp.numpy().copy(), pq.numpy().copy())
            else:
                phi, psi, _ = s.read()
                out[route] = (phi, psi)
    assert np.array_equal(out["pinned"][0], out["pageable"][0])
    assert np.array_equal(out["pinned"][1], out["pageable"][1])
    ref, refq, _ = oracle.run(phi0, phi1, L, mu, lam, bc, 0.0, dt, nsteps)
    tol = 1e-11 if prec == 0 else 2e-5
    phi = out["pinned"][0]
    assert np.max(np.abs(phi - ref)) <= tol * np.max(np.abs(ref))


@pytest.mark.parametrize("pinned", [True, False])
@pytest.mark.parametrize("bc,prec", [(0, 1), (1, 1), (1, 0)])
def test_streamed_solves_equal_each_solved_alone(env, bc, prec, pinned):
    """Streaming host I/O: three problems with different data solved one after
    another on one context, the next problem's data prefetched while the
    current one steps and each phi read back asynchronously while the next
    one starts, end bitwise where each ends solved alone (hbe_set_initial,
    hbe_step, hbe_read).  Any missing order between the copies, the pack,
    the steps and the unpack shows up as another problem's bits."""
    torch, hbe = env
    N, nsteps, mu, lam = 40, 5, 1.2, 0.8

    def host(a):
        a = np.ascontiguousarray(a, dtype=np.float64)
        return torch.from_numpy(a).pin_memory().numpy() if pinned else a

    probs = [rand_problem(N, bc, 30 + k) for k in range(3)]
    L, dt = probs[0][2], probs[0][3]
    inputs = [(host(p[0]), host(p[1])) for p in probs]
    outs = [host(np.zeros((N, N, N))) for _ in range(3)]
    with hbe.Solver(N, L, mu, lam, bc, prec) as s:
        s.set_initial(*inputs[0])
        for k in range(3):
            s.step_async(nsteps, dt)
            if k + 1 < 3:
                s.prefetch_initial(*inputs[k + 1])
            assert s.sync() == hbe.OK
            s.read_async(outs[k])
            if k + 1 < 3:
                s.set_initial_prefetched()
        s.read_wait()
    for k in range(3):
        with hbe.Solver(N, L, mu, lam, bc, prec) as s:
            s.set_initial(probs[k][0], probs[k][1])
            s.step(nsteps, dt)
            ref, _, _ = s.read(psi=False)
        assert np.array_equal(outs[k], ref), k
    assert not np.array_equal(outs[0], outs[1])


def test_prefetched_initial_data_needs_a_prefetch(env):
    torch, hbe = env
    with hbe.Solver(16, 4.0, 1.0, 1.0, 0, hbe.FP32) as s:
        with pytest.raises(hbe._lib.HBEError) as e:
            s.set_initial_prefetched()
        assert e.value.status == hbe._lib.ESTATE
        s.read_wait()  # nothing pending: returns at once
