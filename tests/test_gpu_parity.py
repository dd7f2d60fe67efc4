"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle.

Tolerances (relative max-norm over the N^3 unknowns, C14 reading):
FP64 1e-11, FP32 (compensated state) 2e-5, plain FP32 1e-4, BF16-stored
stage values 5e-3 (bf16 keeps 8 significant bits of each G).
"""
import os
import tempfile

import numpy as np
import pytest

import __graft_entry__  # noqa: F401
import hbe_inputs as hi
import oracle

pytestmark = pytest.mark.gpu

TOL = {0: 1e-11, 1: 2e-5, 2: 5e-3, 3: 1e-4}
PRECS = (0, 1, 2, 3)


@pytest.fixture(scope="module")
def hbe():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_1803_01291_gb300 as m
    return m


def relerr(a, b):
    return np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300)


def solve(hbe, prob, prec, nsteps, variant=0, zchunk=0, t0=0.0):
    with hbe.Solver(prob.N, prob.L, prob.mu, prob.lam, prob.bc, prec) as s:
        s.set_tuning(variant, zchunk)
        s.set_initial(prob.phi0, prob.phi1, t0)
        st = s.step(nsteps, prob.dt)
        phi, psi, t = s.read()
        return st, phi, psi, t


def rand_problem(N, bc, seed, L=12.0, mu=1.1, lam=0.9):
    from scipy import ndimage
    rng = np.random.default_rng(seed)
    mode = "wrap" if bc == 1 else "constant"
    phi0 = ndimage.gaussian_filter(rng.standard_normal((N, N, N)), 2.0, mode=mode) * 4
    phi1 = ndimage.gaussian_filter(rng.standard_normal((N, N, N)), 2.0, mode=mode)
    h = hi.grid_spacing(N, L, bc)
    return hi.Problem(N, L, mu, lam, bc, phi0, phi1, 0.0, h / 4, 0, f"rand{N}")


@pytest.mark.parametrize("prec", PRECS)
def test_radial_bump_64_full_horizon(hbe, prec):
    """64^3 on [-5, 5]^3, mu = lambda = 1, 1.5 exp(-1/(1 - r^2/9)), t in [0, 2]."""
    prob = hi.radial_bump_problem(64)
    ref, refq, _ = oracle.run(prob.phi0, prob.phi1, prob.L, prob.mu, prob.lam, prob.bc, 0.0,
                              prob.dt, prob.nsteps)
    st, phi, psi, t = solve(hbe, prob, prec, prob.nsteps)
    assert st == hbe.OK
    assert abs(t - 2.0) < 1e-12
    assert relerr(phi, ref) <= TOL[prec]
    assert relerr(psi, refq) <= 4 * TOL[prec]


@pytest.mark.parametrize("bc", [0, 1])
@pytest.mark.parametrize("N", [20, 36, 44])
@pytest.mark.parametrize("prec", PRECS)
def test_ragged_sizes(hbe, prec, N, bc):
    """Sizes that are not multiples of the tiles (ragged x, y and z chunks)."""
    prob = rand_problem(N, bc, seed=N + 7 * bc)
    nsteps = 5
    ref, refq, _ = oracle.run(prob.phi0, prob.phi1, prob.L, prob.mu, prob.lam, bc, 0.25, prob.dt,
                              nsteps)
    st, phi, psi, _ = solve(hbe, prob, prec, nsteps, zchunk=7, t0=0.25)
    assert st == hbe.OK
    assert relerr(phi, ref) <= TOL[prec]
    assert relerr(psi, refq) <= 4 * TOL[prec]


@pytest.mark.parametrize("prec", PRECS)
def test_tiling_does_not_change_results(hbe, prec):
    """Every tile variant and z-chunk computes each point with the same
    operations, so all of them agree bit for bit."""
    prob = rand_problem(40, 1, seed=3)
    _, base, baseq, _ = solve(hbe, prob, prec, 3, variant=0, zchunk=0)
    nvar = len(hbe.variants(prec))
    for v in range(nvar):
        for zc in (0, 5, 40):
            _, phi, psi, _ = solve(hbe, prob, prec, 3, variant=v, zchunk=zc)
            assert np.array_equal(phi, base) and np.array_equal(psi, baseq), (v, zc)


def test_octant_symmetry_bitwise(hbe):
    N, L = 32, 10.0
    x = hi.grid_coords(N, L, 0)
    phi0 = (1.2 * np.exp(-x[None, None, :] ** 2 / 2.0) * np.exp(-x[None, :, None] ** 2 / 3.0)
            * np.exp(-x[:, None, None] ** 2 / 1.5))
    prob = hi.Problem(N, L, 1.2, 0.8, 0, phi0, -0.5 * phi0, 0, 0.05, 0)
    for prec in PRECS:
        _, phi, _, _ = solve(hbe, prob, prec, 8)
        for ax in range(3):
            assert np.array_equal(phi, np.flip(phi, axis=ax)), (prec, ax)


def test_periodic_grf_and_shift(hbe):
    prob = hi.grf_problem(32, lam=1.0, seed=0)
    ref, _, _ = oracle.run(prob.phi0, prob.phi1, prob.L, prob.mu, prob.lam, 1, 0.0, prob.dt, 6)
    for prec in PRECS:
        _, phi, _, _ = solve(hbe, prob, prec, 6)
        assert relerr(phi, ref) <= TOL[prec]
    # an integer-cell shift of periodic data shifts the solution bit for bit
    sh = (5, -3, 11)
    moved = hi.Problem(prob.N, prob.L, prob.mu, prob.lam, 1, np.roll(prob.phi0, sh, (0, 1, 2)),
                       np.roll(prob.phi1, sh, (0, 1, 2)), 0, prob.dt, 0)
    for prec in PRECS:
        _, a, _, _ = solve(hbe, prob, prec, 4)
        _, b, _, _ = solve(hbe, moved, prec, 4)
        assert np.array_equal(b, np.roll(a, sh, (0, 1, 2))), prec


def test_homogeneous_blowup_stops_like_oracle(hbe):
    """Periodic homogeneous data in the focusing case: stop after the first
    step with max|phi| > 1e6, same step as the oracle."""
    N, dt = 8, 1e-2
    a0 = 3.0 / np.e
    phi0, phi1 = np.full((N, N, N), a0), np.zeros((N, N, N))
    _, _, n_ref = oracle.run(phi0, phi1, 4.0, 1.0, -1.0, 1, 0.0, dt, 100000, stop_threshold=1e6)
    for prec in (0, 1):
        with hbe.Solver(N, 4.0, 1.0, -1.0, 1, prec) as s:
            s.set_initial(phi0, phi1)
            s.set_stop(1e6)
            st = s.step(1000, dt)
            n, t = s.progress()
            assert st == hbe.STOPPED
            assert n == n_ref
            assert abs(t - n_ref * dt) < 1e-12
            assert s.diag()["max_abs_phi"] > 1e6


def test_nonfinite_stops(hbe):
    N = 16
    phi0 = np.zeros((N, N, N))
    phi0[3, 4, 5] = np.nan
    with hbe.Solver(N, 4.0, 1.0, 1.0, 0, 1) as s:
        s.set_initial(phi0, np.zeros_like(phi0))
        assert s.step(20, 0.01) == hbe.NONFINITE
        assert s.progress()[0] == 1
        assert not s.diag()["finite"]


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("bc", [0, 1])
def test_diag_masks_bit_exact(hbe, prec, bc):
    """Sign masks and component counts of the GPU's own field equal the
    oracle's on that same field."""
    prob = rand_problem(40, bc, seed=11 + bc)
    with hbe.Solver(prob.N, prob.L, prob.mu, prob.lam, bc, prec) as s:
        s.set_initial(prob.phi0, prob.phi1)
        s.step(3, prob.dt)
        phi, _, _ = s.read(psi=False)
        for eps in (0.0, 0.05):
            g = s.diag(eps=eps, masks=True)
            o = oracle.diag(phi, bc, eps=eps)
            assert np.array_equal(g["pos_mask"], o["pos_mask"])
            assert np.array_equal(g["neg_mask"], o["neg_mask"])
            for k in ("n_pos", "n_neg", "bubble_count", "finite"):
                assert g[k] == o[k], k
            assert g["max_abs_phi"] == o["max_abs_phi"]


def test_save_load_resumes_bitwise(hbe):
    prob = rand_problem(36, 0, seed=5)
    for prec in PRECS:
        with hbe.Solver(prob.N, prob.L, prob.mu, prob.lam, 0, prec) as a:
            a.set_initial(prob.phi0, prob.phi1)
            a.step(7, prob.dt)
            full, fullq, _ = a.read()
        with hbe.Solver(prob.N, prob.L, prob.mu, prob.lam, 0, prec) as b:
            b.set_initial(prob.phi0, prob.phi1)
            b.step(3, prob.dt)
            with tempfile.TemporaryDirectory() as d:
                path = os.path.join(d, "ck.bin")
                b.save(path)
                with hbe.Solver(prob.N, prob.L, prob.mu, prob.lam, 0, prec) as c:
                    c.load(path)
                    c.step(4, prob.dt)
                    phi, psi, _ = c.read()
        assert np.array_equal(phi, full) and np.array_equal(psi, fullq), prec


def test_split_steps_equal_one_call(hbe):
    """t_n = t0 + n dt: 3 + 9 steps in two calls equal 12 in one, bitwise."""
    prob = rand_problem(24, 1, seed=9)
    for prec in (0, 1):
        _, a, aq, _ = solve(hbe, prob, prec, 12)
        with hbe.Solver(prob.N, prob.L, prob.mu, prob.lam, 1, prec) as s:
            s.set_initial(prob.phi0, prob.phi1)
            s.step(3, prob.dt)
            s.step(9, prob.dt)
            b, bq, _ = s.read()
        assert np.array_equal(a, b) and np.array_equal(aq, bq)


def test_partial_replays_launch_only_taken_steps(hbe):
    """A call whose step count is not a multiple of the graph length K = 8
    ends with a graph of the remaining steps: 11 steps launch 11 steps' worth
    of kernels (2 stage pairs + 2 periodic ghost copies each), and 11 calls of
    one step (11 one-step graphs) give the same bits as one call of 11."""
    prob = rand_problem(28, 1, seed=21)
    for prec in (0, 1):
        with hbe.Solver(prob.N, prob.L, prob.mu, prob.lam, 1, prec) as s:
            s.set_initial(prob.phi0, prob.phi1)
            l0 = s.launches
            s.step(11, prob.dt)
            assert s.launches - l0 == 11 * 4
            a, aq, _ = s.read()
        with hbe.Solver(prob.N, prob.L, prob.mu, prob.lam, 1, prec) as s:
            s.set_initial(prob.phi0, prob.phi1)
            for _ in range(11):
                s.step(1, prob.dt)
            b, bq, _ = s.read()
        assert np.array_equal(a, b) and np.array_equal(aq, bq)


def test_batch_alone_equals_mixed(hbe):
    """Members of a batch (mixed sizes, parameters, step counts) end bit for
    bit where they end when stepped alone."""
    rng = np.random.default_rng(0)
    reqs = [r for r in hi.request_stream(10, seed=1, sizes=(32, 48, 64))]
    alone = {}
    for r in reqs:
        phi0, phi1 = r.initial()
        n, dt = r.steps()
        n = min(n, 20 + r.rid)
        with hbe.Solver(r.N, r.L, r.mu, r.lam, 0, hbe.FP32) as s:
            s.set_initial(phi0, phi1)
            s.step(n, dt)
            alone[r.rid] = s.read()[0]
    b = hbe.Batch(hbe.FP32, K=4)
    solvers = {}
    pending = list(reqs)
    finished = {}
    # admit in waves to exercise joins while others are running
    while pending or len(b):
        for _ in range(int(rng.integers(1, 4))):
            if pending:
                r = pending.pop(0)
                phi0, phi1 = r.initial()
                n, dt = r.steps()
                n = min(n, 20 + r.rid)
                s = hbe.Solver(r.N, r.L, r.mu, r.lam, 0, hbe.FP32)
                s.set_initial(phi0, phi1)
                solvers[id(s)] = (r, s)
                b.add(s, n, dt)
        for s in b.run():
            r, _ = solvers[id(s)]
            finished[r.rid] = s.read()[0]
            s.close()
    assert sorted(finished) == sorted(alone)
    for rid in alone:
        assert np.array_equal(finished[rid], alone[rid]), rid


@pytest.mark.parametrize("prec", [0, 1])
def test_batch_with_periodic_members_equals_alone(hbe, prec):
    """Periodic and zero-Dirichlet members in one batch (ragged sizes, their
    own step counts): the batched graph's ghost copies serve the periodic
    members, and every member ends bit for bit where it ends alone."""
    cases = [(24, 1, 7), (40, 0, 9), (36, 1, 12), (64, 1, 5), (20, 0, 11), (44, 1, 8)]
    probs = [rand_problem(N, bc, seed=10 + i) for i, (N, bc, _) in enumerate(cases)]
    alone = []
    for prob, (_, _, n) in zip(probs, cases):
        with hbe.Solver(prob.N, prob.L, prob.mu, prob.lam, prob.bc, prec) as s:
            s.set_initial(prob.phi0, prob.phi1)
            s.step(n, prob.dt)
            alone.append(s.read()[:2])
    b = hbe.Batch(prec, K=4)
    solvers = []
    for i, (prob, (_, _, n)) in enumerate(zip(probs, cases)):
        s = hbe.Solver(prob.N, prob.L, prob.mu, prob.lam, prob.bc, prec)
        s.set_initial(prob.phi0, prob.phi1)
        solvers.append(s)
        if i < 3:
            b.add(s, n, prob.dt)
    done = {}
    later = list(range(3, len(cases)))
    while len(b) or later:
        for s in b.run():
            done[solvers.index(s)] = s.read()[:2]
        if later:  # joins while others are running
            i = later.pop(0)
            b.add(solvers[i], cases[i][2], probs[i].dt)
    b.close()
    for s in solvers:
        s.close()
    assert sorted(done) == list(range(len(cases)))
    for i in range(len(cases)):
        assert np.array_equal(done[i][0], alone[i][0]), i
        assert np.array_equal(done[i][1], alone[i][1]), i


@pytest.mark.parametrize("schedule", [0, 1])
@pytest.mark.parametrize("prec", PRECS)
def test_periodic_ghosts_under_nan_canary(hbe, prec, schedule, monkeypatch):
    """With HBE_DEBUG_NAN_GHOSTS every field of a periodic context starts as NaN,
    so a ghost cell read before the ghost-copy launch refreshed it would make
    the result non-finite.  Ragged sizes, both schedules, several steps: the
    result stays finite and within tolerance of the oracle."""
    monkeypatch.setenv("HBE_DEBUG_NAN_GHOSTS", "1")
    for N in (20, 36):
        prob = rand_problem(N, 1, seed=N)
        nsteps = 4
        ref, _, _ = oracle.run(prob.phi0, prob.phi1, prob.L, prob.mu, prob.lam, 1, 0.0, prob.dt,
                               nsteps)
        with hbe.Solver(prob.N, prob.L, prob.mu, prob.lam, 1, prec) as s:
            s.set_schedule(schedule)
            s.set_initial(prob.phi0, prob.phi1)
            st = s.step(nsteps, prob.dt)
            phi, psi, _ = s.read()
        assert st == hbe.OK
        assert np.all(np.isfinite(phi)) and np.all(np.isfinite(psi))
        assert relerr(phi, ref) <= TOL[prec]


def test_errors_are_returned_not_raised_by_the_library(hbe):
    with pytest.raises(hbe.HBEError):
        hbe.Solver(4, 1.0, 1.0, 1.0)
    with hbe.Solver(16, 4.0, 1.0, 1.0) as s:
        with pytest.raises(hbe.HBEError):
            s.step(1, 0.01)  # no initial data
        s.set_initial(np.zeros((16,) * 3), np.zeros((16,) * 3))
        with pytest.raises(hbe.HBEError):
            s.step(1, -1.0)
        with pytest.raises(hbe.HBEError):
            s.set_tuning(99, 0)
