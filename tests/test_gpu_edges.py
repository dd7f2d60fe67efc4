"""Edge cases through the C ABI: zero steps, the smallest grid the library
accepts, a grid too large for the device (a clean HBE_ENOMEM, the library
still usable afterwards), a stage kernel whose bounded wait runs out (a clean
HBE_ETIMEOUT), and the largest FP32 grid that fits on one GB300, checked by an
invariant that holds at any size (data even in x, y and z on the symmetric
grid of Sec. 2.1 stays even, bit for bit)."""
import ctypes
import time

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


def rand_fields(N, bc, seed):
    from scipy import ndimage
    rng = np.random.default_rng(seed)
    mode = "wrap" if bc == 1 else "constant"
    a = ndimage.gaussian_filter(rng.standard_normal((N, N, N)), 1.5, mode=mode) * 3
    b = ndimage.gaussian_filter(rng.standard_normal((N, N, N)), 1.5, mode=mode)
    return a, b


@pytest.mark.parametrize("prec", [0, 1, 2, 3])
def test_zero_steps_return_the_initial_data(hbe, prec):
    N = 20
    phi0, phi1 = rand_fields(N, 0, 1)
    with hbe.Solver(N, 8.0, 1.0, 1.0, 0, prec) as s:
        s.set_initial(phi0, phi1, 0.25)
        assert s.step(0, 0.01) == hbe.OK
        phi, psi, t = s.read()
    assert t == 0.25
    if prec == hbe.FP64:
        assert np.array_equal(phi, phi0) and np.array_equal(psi, phi1)
    elif prec in (hbe.FP32, hbe.BF16):  # (hi, lo) float pairs hold the doubles to ~2^-48
        assert np.max(np.abs(phi - phi0)) <= 1e-14 * np.max(np.abs(phi0))
        assert np.max(np.abs(psi - phi1)) <= 1e-14 * np.max(np.abs(phi1))
    else:
        assert np.array_equal(phi, phi0.astype(np.float32).astype(np.float64))


@pytest.mark.parametrize("bc", [0, 1])
@pytest.mark.parametrize("prec,tol", [(0, 1e-11), (1, 2e-5)])
def test_smallest_grid_matches_oracle(hbe, bc, prec, tol):
    N, L, mu, lam, n = 8, 4.0, 1.2, 0.8, 7
    phi0, phi1 = rand_fields(N, bc, 2 + bc)
    dt = hi.grid_spacing(N, L, bc) / 4
    with hbe.Solver(N, L, mu, lam, bc, prec) as s:
        s.set_initial(phi0, phi1)
        assert s.step(n, dt) == hbe.OK
        phi, psi, _ = s.read()
    ref, refq, _ = oracle.run(phi0, phi1, L, mu, lam, bc, 0.0, dt, n)
    assert np.max(np.abs(phi - ref)) <= tol * np.max(np.abs(ref))
    assert np.max(np.abs(psi - refq)) <= tol * np.max(np.abs(refq))


def test_sizes_outside_the_limits_are_refused(hbe):
    lib = hbe._lib.load()
    ctx = ctypes.c_void_p()
    assert lib.hbe_create(7, 4.0, 1.0, 1.0, 0, hbe.FP32, ctypes.byref(ctx)) == hbe._lib.EINVAL
    assert lib.hbe_create(2049, 4.0, 1.0, 1.0, 0, hbe.FP32, ctypes.byref(ctx)) == hbe._lib.EINVAL


def test_grid_larger_than_the_device_fails_cleanly(hbe):
    """2048^3 with FP32 compensated state needs 11 fields of 34.6 GB (380 GB):
    creation returns HBE_ENOMEM and the library keeps working."""
    import torch
    lib = hbe._lib.load()
    need = hbe.workspace_bytes(2048, 0, hbe.FP32)
    free, _ = torch.cuda.mem_get_info()
    if need <= free:
        pytest.skip("this device could hold the 2048^3 FP32 problem")
    ctx = ctypes.c_void_p()
    st = lib.hbe_create(2048, 20.0, 1.0, 1.0, 0, hbe.FP32, ctypes.byref(ctx))
    assert st == hbe._lib.ENOMEM and not ctx.value
    test_smallest_grid_matches_oracle(hbe, 0, 1, 2e-5)


def test_withheld_plane_times_out_cleanly(hbe, monkeypatch):
    """With HBE_DEBUG_WITHHOLD_PLANE set at creation, the stages 1+2 producer
    of block 0 never issues the first plane of its first work item: its
    consumers wait on a barrier that nothing completes, give up after their
    bound (~2 s), and the step returns HBE_ETIMEOUT instead of hanging.  The
    library keeps working: a new context matches the oracle."""
    monkeypatch.setenv("HBE_DEBUG_WITHHOLD_PLANE", "1")
    N = 16
    phi0, phi1 = rand_fields(N, 0, 5)
    s = hbe.Solver(N, 4.0, 1.0, 1.0, 0, hbe.FP32)
    try:
        s.set_initial(phi0, phi1)
        t0 = time.perf_counter()
        with pytest.raises(hbe._lib.HBEError) as e:
            s.step(1, hi.grid_spacing(N, 4.0, 0) / 4)
        waited = time.perf_counter() - t0
    finally:
        s.close()
    assert e.value.status == hbe._lib.ETIMEOUT
    assert 1.0 < waited < 60.0
    monkeypatch.delenv("HBE_DEBUG_WITHHOLD_PLANE")
    test_smallest_grid_matches_oracle(hbe, 0, 1, 2e-5)


def test_largest_fp32_grid_keeps_octant_symmetry(hbe):
    """1536^3 (161 GB of fields) from a centred bump built on the device, 3 RK4
    steps: the solution stays even about the centre in x, y and z, bit for
    bit, and finite."""
    import torch
    N = 1536
    need = hbe.workspace_bytes(N, 0, hbe.FP32) + 2 * N ** 3 * 8  # fields, phi and a flip
    free, _ = torch.cuda.mem_get_info()
    if need > 0.9 * free:
        pytest.skip("not enough device memory for the 1536^3 FP32 problem")
    L, dt = 20.0, hi.grid_spacing(N, 20.0, 0) / 4
    with hbe.Solver(N, L, 1.0, 1.0, 0, hbe.FP32) as s:
        s.set_initial_bumps([(1.5, 4.0, (0.0, 0.0, 0.0))])
        assert s.step(3, dt) == hbe.OK
        phi, _ = s.read_device()
        assert bool(torch.isfinite(phi).all())
        assert float(phi.abs().max()) > 0.1
        for ax in range(3):
            assert torch.equal(phi, phi.flip(ax)), ax
        del phi
    torch.cuda.empty_cache()
