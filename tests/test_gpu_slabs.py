"""k virtual z-slabs on one GPU: the halo planes exchanged after each stage
pair make the slabs compute exactly what the undivided grid computes, so the
results are the same bits (FP64 and FP32 with compensated state, both
boundaries, k = 1, 2, 3, 4, step counts that leave a partial graph replay)."""
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
    a = ndimage.gaussian_filter(rng.standard_normal((N, N, N)), 2.0, mode=mode) * 4
    b = ndimage.gaussian_filter(rng.standard_normal((N, N, N)), 2.0, mode=mode)
    return a, b


@pytest.mark.parametrize("bc", [0, 1])
@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("k", [1, 2, 4])
def test_slabs_equal_undivided_grid_bitwise(hbe, bc, prec, k):
    from paper_1803_01291_gb300.slabs import SlabSolver
    N, L, mu, lam, nsteps = 40, 12.0, 1.1, 0.9, 11
    phi0, phi1 = rand_fields(N, bc, 3 + bc)
    dt = hi.grid_spacing(N, L, bc) / 4
    with hbe.Solver(N, L, mu, lam, bc, prec) as s:
        s.set_initial(phi0, phi1)
        assert s.step(nsteps, dt) == hbe.OK
        ref, refq, tref = s.read()
    with SlabSolver(N, L, mu, lam, bc, prec, k=k) as sl:
        sl.set_initial(phi0, phi1)
        assert sl.step(5, dt) == hbe.OK
        assert sl.step(nsteps - 5, dt) == hbe.OK
        phi, psi, t = sl.read()
    assert t == tref
    assert np.array_equal(phi, ref) and np.array_equal(psi, refq)


def test_slabs_ragged_split_matches_oracle(hbe):
    """N = 37 over k = 3 slabs (13, 12, 12 planes) against the oracle."""
    from paper_1803_01291_gb300.slabs import SlabSolver
    N, L, mu, lam, nsteps = 37, 10.0, 1.3, 1.2, 6
    for bc in (0, 1):
        phi0, phi1 = rand_fields(N, bc, 9)
        dt = hi.grid_spacing(N, L, bc) / 4
        with SlabSolver(N, L, mu, lam, bc, hbe.FP64, k=3) as sl:
            sl.set_initial(phi0, phi1)
            sl.step(nsteps, dt)
            phi, _, _ = sl.read()
        ref, _, _ = oracle.run(phi0, phi1, L, mu, lam, bc, 0.0, dt, nsteps)
        assert np.max(np.abs(phi - ref)) <= 1e-11 * np.max(np.abs(ref))
