"""Host-side logic that needs no GPU: the bench's byte model and aggregation,
the autotuner's selection and cache, the server's admission (memory budget,
FIFO order, requeue after an allocation failure) with stand-ins for the
device objects, and the seeded request stream."""
import ctypes
import json
import math

import numpy as np
import pytest

import __graft_entry__  # noqa: F401
import bench
import hbe_inputs as hi
from paper_1803_01291_gb300 import _lib


# ---------------------------------------------------------------- bench byte model
def test_stage_bytes_match_the_design_table():
    one = {"fp64": 80, "fp32": 56, "bf16": 48, "fp32_plain": 40}
    zero = {"fp64": 152, "fp32": 92, "bf16": 74, "fp32_plain": 76}
    for prec in one:
        assert sum(bench.stage_bytes(prec, 1)) == one[prec]
        assert sum(bench.stage_bytes(prec, 0)) == zero[prec]
    assert bench.stage_bytes("fp32", 1) == [16, 40]


def test_aggregate_is_all_units_over_the_slowest_rank():
    assert bench.aggregate(2e9, 0.5, 4) == pytest.approx(16.0)


# ---------------------------------------------------------------- autotuner
def test_autotune_picks_the_fastest_and_caches_it(tmp_path, monkeypatch):
    from paper_1803_01291_gb300 import autotune
    monkeypatch.setenv("HBE_AUTOTUNE_CACHE", str(tmp_path / "c.json"))
    monkeypatch.setattr(autotune, "_gpu_name", lambda: "test-gpu")
    nvar = len(autotune.variants(_lib.FP32))

    def fake(N, bc, prec, v, zc, steps=10, warmup=3, seed=0, schedule=1):
        # fastest: schedule 0, variant nvar - 1, the second z-chunk candidate
        zcs = list(autotune.zchunk_candidates(N))
        return 1.0 + (0 if schedule == 0 else 0.5) + (nvar - 1 - v) * 0.1 + \
            (0 if zc == zcs[1] else 0.05)

    monkeypatch.setattr(autotune, "measure", fake)
    e = autotune.tune(96, 0, _lib.FP32)
    assert (e["variant"], e["zchunk"], e["schedule"]) == \
        (nvar - 1, list(autotune.zchunk_candidates(96))[1], 0)
    assert len(e["sweep"]) == 2 * nvar * len(list(autotune.zchunk_candidates(96)))
    cache = json.load(open(tmp_path / "c.json"))
    assert list(cache) == ["test-gpu|N=96|bc=0|prec=fp32"]
    assert autotune.best(96, 0, _lib.FP32) == (e["variant"], e["zchunk"], 0)
    assert autotune.best(97, 0, _lib.FP32) == (0, 0, 1)  # nothing cached: library defaults


def test_zchunk_candidates_cover_whole_and_split_columns():
    c = list(autotune_mod().zchunk_candidates(512))
    assert c[0] == 0 and 512 in c and all(z >= 16 or z == 0 for z in c)
    assert c == sorted(set(c))


def autotune_mod():
    from paper_1803_01291_gb300 import autotune
    return autotune


# ---------------------------------------------------------------- server admission
class FakeSolver:
    created = 0
    fail_at = None
    live = 0

    def __init__(self, N, L, mu, lam, bc, prec):
        FakeSolver.created += 1
        if FakeSolver.created == FakeSolver.fail_at:
            raise _lib.HBEError(_lib.ENOMEM, "injected")
        self.N, self.steps, self.target = N, 0, 0
        self.handle = ctypes.c_void_p(1000 + FakeSolver.created)
        FakeSolver.live += 1

    def set_tuning(self, v, zc):
        self.variant = v

    def set_initial_bumps(self, bumps):
        pass

    def sync(self):
        return _lib.OK

    def set_stream(self, stream):
        pass

    def progress(self):
        return self.steps, 0.0

    def diag(self):
        return {"max_abs_phi": float(self.N)}

    def close(self):
        FakeSolver.live -= 1


class FakeBatch:
    def __init__(self, prec, K):
        self.K, self.members, self.launches = K, [], 0
        self.max_seen = 0
        self.in_flight = False

    def add(self, s, nsteps, dt):
        assert not self.in_flight, "add with a run in flight"
        s.target = nsteps
        self.members.append(s)
        self.max_seen = max(self.max_seen, len(self.members))

    def launch(self):
        assert not self.in_flight, "launch with a run in flight"
        for s in self.members:
            s.steps = min(s.target, s.steps + self.K)
        self.launches += 2 * self.K
        self.in_flight = True

    def collect(self):
        if not self.in_flight:
            return []
        self.in_flight = False
        done = [s for s in self.members if s.steps >= s.target]
        self.members = [s for s in self.members if s.steps < s.target]
        return done

    def run(self):
        self.launch()
        return self.collect()

    def __len__(self):
        return len(self.members)

    def close(self):
        pass


@pytest.fixture
def server_mod(monkeypatch):
    from paper_1803_01291_gb300 import serve
    FakeSolver.created, FakeSolver.fail_at, FakeSolver.live = 0, None, 0
    monkeypatch.setattr(serve, "Solver", FakeSolver)
    monkeypatch.setattr(serve, "Batch", FakeBatch)
    return serve


def _requests(serve, sizes, nsteps=20):
    return [serve.SolveRequest(i, 0.001 * i, N, 20.0, 1.0, 1.0, T=nsteps * 0.01, dt=0.01,
                               bumps=[(1.0, 2.0, (0.0, 0.0, 0.0))])
            for i, N in enumerate(sizes)]


def test_admission_respects_the_memory_budget(server_mod):
    serve = server_mod
    reqs = _requests(serve, [64, 48, 64, 32, 64, 48])
    need = serve.workspace_bytes(64, 0, _lib.FP32)
    srv = serve.Server(_lib.FP32, K=4, hbm_budget=2 * need)
    stats = srv.run(reqs, realtime=False)
    assert sorted(r.rid for r in stats.results) == list(range(len(reqs)))
    assert stats.peak_bytes <= 2 * need
    assert all(r.steps == 20 for r in stats.results)
    assert FakeSolver.live == 0  # every member released
    # closed loop: every request counts as arrived at time 0
    assert all(r.arrival == 0.0 for r in stats.results)


def test_requeue_after_allocation_failure(server_mod):
    serve = server_mod
    FakeSolver.fail_at = 3
    reqs = _requests(serve, [32, 32, 32, 32])
    srv = serve.Server(_lib.FP32, K=4, hbm_budget=1 << 40)
    stats = srv.run(reqs, realtime=False)
    assert stats.admission_retries == 1
    assert sorted(r.rid for r in stats.results) == [0, 1, 2, 3]


def test_allocation_failure_with_nothing_to_wait_for_raises(server_mod):
    serve = server_mod
    FakeSolver.fail_at = 1
    srv = serve.Server(_lib.FP32, K=4, hbm_budget=1 << 40)
    with pytest.raises(_lib.HBEError):
        srv.run(_requests(serve, [32]), realtime=False)


def test_request_larger_than_the_budget_is_refused(server_mod):
    serve = server_mod
    srv = serve.Server(_lib.FP32, K=4, hbm_budget=1000)
    with pytest.raises(ValueError):
        srv.run(_requests(serve, [64]), realtime=False)


def test_every_size_shares_one_variant_by_default(server_mod):
    """Without a tuning callback all members use variant 0, so a batch graph
    launches one pair of stage kernels per step; a callback overrides it."""
    serve = server_mod
    srv = serve.Server(_lib.FP32, K=4, hbm_budget=1 << 40)
    assert {srv._default_variant(N) for N in (32, 64, 192, 256)} == {0}
    reqs = _requests(serve, [32, 64])
    srv.run(reqs, realtime=False)
    srv2 = serve.Server(_lib.FP32, K=4, hbm_budget=1 << 40, tuning=lambda N, p: (3, 0))
    seen = []
    orig = FakeSolver.set_tuning
    FakeSolver.set_tuning = lambda self, v, zc: seen.append(v)
    try:
        srv2.run(_requests(serve, [32]), realtime=False)
    finally:
        FakeSolver.set_tuning = orig
    assert seen == [3]


def test_server_uses_the_autotuner_cache(server_mod, tmp_path, monkeypatch):
    """Sizes the autotuner has tuned get its (variant, z-chunk); others variant 0."""
    serve = server_mod
    from paper_1803_01291_gb300 import autotune
    monkeypatch.setenv("HBE_AUTOTUNE_CACHE", str(tmp_path / "c.json"))
    monkeypatch.setattr(autotune, "_gpu_name", lambda: "test-gpu")
    cache = {autotune._key(48, 0, _lib.FP32): {"variant": 2, "zchunk": 16, "schedule": 0}}
    autotune.save_cache(cache)
    seen = []
    orig = FakeSolver.set_tuning
    FakeSolver.set_tuning = lambda self, v, zc: seen.append((self.N, v, zc))
    try:
        srv = serve.Server(_lib.FP32, K=4, hbm_budget=1 << 40)
        srv.run(_requests(serve, [48, 64, 48]), realtime=False)
    finally:
        FakeSolver.set_tuning = orig
    assert sorted(seen) == [(48, 2, 16), (48, 2, 16), (64, 0, 0)]


# ---------------------------------------------------------------- request stream
def test_request_stream_is_seeded_and_in_range():
    a = hi.request_stream(50, seed=3)
    b = hi.request_stream(50, seed=3)
    assert [(r.N, r.mu, r.lam, r.T) for r in a] == [(r.N, r.mu, r.lam, r.T) for r in b]
    assert all(r.N in hi.SERVE_SIZES for r in a)
    assert all(0.5 <= r.mu <= 2 and 0.5 <= r.lam <= 2 and 1 <= r.T <= 6 for r in a)
    assert all(1 <= len(r.bumps) <= 4 for r in a)
    assert np.all(np.diff([r.arrival for r in a]) > 0)
    for r in a[:5]:
        n, dt = r.steps()
        h = hi.grid_spacing(r.N, r.L, 0)
        assert dt <= h / 4 + 1e-15 and abs(n * dt - r.T) < 1e-9


# ---------------------------------------------------------------- reference arm
def _ref_args(N=64):
    import argparse
    return argparse.Namespace(N=N, steps=1, warmup=3, gpus=1)


def test_reference_arm_prints_one_oracle_line(monkeypatch, capsys):
    """`bench.py --impl reference`: the CPU oracle timed on a slab of the same
    workload, one JSON line with the contract's keys."""
    monkeypatch.setenv("RANK", "0")
    bench.reference_arm(_ref_args())
    lines = [ln for ln in capsys.readouterr().out.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    line = json.loads(lines[0])
    assert line["impl"] == "reference" and line["metric"] == bench.METRIC
    assert line["value"] > 0 and line["unit"] == "Gpoint-steps/s"
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["value"] == line["value"]
    assert line["e2e"] == {"value": line["value"], "unit": "Gpoint-steps/s",
                           "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert line["config"]["workload"] == "hbe-512-periodic-grf" and line["config"]["N"] == 64


def test_reference_arm_is_silent_on_other_ranks(monkeypatch, capsys):
    monkeypatch.setenv("RANK", "1")
    bench.reference_arm(_ref_args())
    assert capsys.readouterr().out == ""


# ---------------------------------------------------------------- end-to-end harness
class _Buf:
    def __init__(self):
        import numpy as _np
        self.a = _np.zeros((2, 2, 2))

    def numpy(self):
        return self.a

    def data_ptr(self):
        return 0


def test_pipelined_e2e_moves_every_solve_inside_the_timed_region():
    """bench.e2e_solve_pipelined on a recording fake: every solve gets its
    inputs (direct for the first, prefetched for the others), steps and sends
    phi back (async for all but the last, direct for the last); each prefetch
    is issued while a solve's steps are in flight (between step_async and
    sync), each async read right after a solve's sync (its copy then overlaps
    the next solve), and nothing is left pending when the clock stops."""
    log = []

    class Lib:
        def hbe_read(self, *a):
            log.append("read_direct")

    class FakeSolver:
        def __init__(self, *a):
            self.lib, self.handle, self.stepping = Lib(), None, False

        def set_initial(self, a, b):
            log.append("set_initial")

        def prefetch_initial(self, a, b):
            log.append("prefetch" + ("*" if self.stepping else ""))

        def set_initial_prefetched(self, t0=0.0):
            log.append("set_prefetched")

        def step(self, n, dt):
            log.append("step")

        def step_async(self, n, dt):
            self.stepping = True
            log.append("step_async")

        def sync(self):
            self.stepping = False
            log.append("sync")
            return 0

        def read_async(self, o):
            log.append("read_async")

        def read_wait(self):
            log.append("read_wait")

        def close(self):
            log.append("close")

    class FakeHbe:
        Solver = FakeSolver

    class FakeTorch:
        class cuda:
            @staticmethod
            def synchronize():
                log.append("cuda_sync")

    class Prob:
        N, L, mu, lam, bc, dt = 2, 1.0, 1.0, 1.0, 0, 0.1

    solves = 4
    total, st, _, phases = bench.e2e_solve_pipelined(FakeHbe, FakeTorch, Prob, 1, 3, solves,
                                                     (_Buf(), _Buf(), _Buf()))
    timed = log[log.index("cuda_sync") + 1:]
    assert len(phases) == solves and st == 0 and total >= 0
    assert timed.count("step_async") == solves
    assert timed[0] == "set_initial"                        # the first inputs: direct
    assert timed.count("set_prefetched") == solves - 1       # the others: prefetched
    assert timed.count("prefetch*") == solves - 1            # ... while a solve steps
    assert "prefetch" not in timed
    assert timed.count("read_async") == solves - 1           # phi of all but the last: async
    assert timed[-3:] == ["read_wait", "read_direct", "close"]  # last phi direct, none pending
    for k in range(solves - 1):                              # async reads follow a sync
        i = [j for j, e in enumerate(timed) if e == "read_async"][k]
        assert timed[i - 1] == "sync"
