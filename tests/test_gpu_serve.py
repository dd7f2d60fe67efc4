"""Continuous-batching server: every request completes, memory admission is
respected, and each result equals the same problem solved alone (bitwise)."""
import numpy as np
import pytest

import __graft_entry__  # noqa: F401
import hbe_inputs as hi

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hbe():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_1803_01291_gb300 as m
    return m


def small_stream(count, seed):
    reqs = hi.request_stream(count, seed=seed, rate=200.0, sizes=(32, 48, 64))
    for r in reqs:
        r.T = min(r.T, 0.6)  # short horizons keep the test quick
    return reqs


def test_bump_initial_data_matches_host_generator(hbe):
    r = small_stream(1, 5)[0]
    phi0, _ = r.initial()
    for prec, tol in ((hbe.FP64, 4e-16), (hbe.FP32, 0.0)):
        with hbe.Solver(r.N, r.L, r.mu, r.lam, 0, prec) as s:
            s.set_initial_bumps(r.bumps)
            a = s.read()[0]
        ref = phi0 if prec == hbe.FP64 else phi0.astype(np.float32).astype(np.float64)
        if prec == hbe.FP32:
            # hi + lo pair holds the double to ~2^-48 relative
            assert np.max(np.abs(a - phi0)) <= 1e-14 * max(1.0, np.max(np.abs(phi0)))
        else:
            assert np.max(np.abs(a - ref)) <= tol * max(1.0, np.max(np.abs(ref))) * 8


@pytest.mark.parametrize("realtime", [False, True])
def test_server_completes_and_matches_alone(hbe, realtime):
    from paper_1803_01291_gb300 import serve
    reqs = serve.requests_from_stream(small_stream(10, 7))
    budget = 3 * hbe.workspace_bytes(64, 0, hbe.FP32)
    srv = serve.Server(hbe.FP32, K=4, hbm_budget=budget)
    stats = srv.run(reqs, realtime=realtime)
    srv.close()
    assert len(stats.results) == len(reqs)
    assert stats.peak_bytes <= budget
    assert stats.peak_members >= 1
    summ = stats.summary()
    assert summ["p99_latency_s"] >= summ["p50_latency_s"] >= 0
    by_id = {r.rid: r for r in stats.results}
    for q in reqs:
        res = by_id[q.rid]
        assert res.steps == q.nsteps
        with hbe.Solver(q.N, q.L, q.mu, q.lam, 0, hbe.FP32) as s:
            s.set_initial_bumps(q.bumps)
            s.step(q.nsteps, q.dt)
            assert s.diag()["max_abs_phi"] == res.max_abs_phi


def test_alone_baseline_runs(hbe):
    from paper_1803_01291_gb300 import serve
    reqs = serve.requests_from_stream(small_stream(3, 9))
    out = serve.run_alone(reqs, hbe.FP64)
    assert out["requests"] == 3 and out["gpoint_steps_per_s"] > 0


def test_server_requeues_after_allocation_failure(hbe, monkeypatch):
    """Failure detection, injected on the host: the third context creation
    fails with HBE_ENOMEM (HBE_FAULT=alloc:3).  The server keeps the request,
    runs the batch it has, admits it later, and every result is still the
    problem's result alone."""
    from paper_1803_01291_gb300 import serve
    reqs = serve.requests_from_stream(small_stream(6, 11))
    monkeypatch.setenv("HBE_FAULT", "alloc:3")
    srv = serve.Server(hbe.FP32, K=4)
    stats = srv.run(reqs, realtime=False)
    srv.close()
    monkeypatch.delenv("HBE_FAULT")
    assert stats.admission_retries == 1
    assert sorted(r.rid for r in stats.results) == sorted(q.rid for q in reqs)
    by_id = {r.rid: r for r in stats.results}
    for q in reqs:
        with hbe.Solver(q.N, q.L, q.mu, q.lam, 0, hbe.FP32) as s:
            s.set_initial_bumps(q.bumps)
            s.step(q.nsteps, q.dt)
            assert s.diag()["max_abs_phi"] == by_id[q.rid].max_abs_phi


def test_server_fields_equal_alone_bitwise(hbe):
    """Every request's final phi, read through the server (keep_fields), is
    the same bits as the problem solved alone: the batched runner, the
    pipelined runs and the side-stream retirement change nothing."""
    from paper_1803_01291_gb300 import serve
    reqs = serve.requests_from_stream(small_stream(8, 13))
    srv = serve.Server(hbe.FP32, K=4, keep_fields=True)
    stats = srv.run(reqs, realtime=False)
    srv.close()
    by_id = {r.rid: r for r in stats.results}
    assert sorted(by_id) == sorted(q.rid for q in reqs)
    for q in reqs:
        res = by_id[q.rid]
        assert res.phi is not None and res.steps == q.nsteps
        with hbe.Solver(q.N, q.L, q.mu, q.lam, 0, hbe.FP32) as s:
            s.set_initial_bumps(q.bumps)
            s.step(q.nsteps, q.dt)
            alone = s.read(psi=False)[0]
        assert np.array_equal(res.phi, alone), q.rid


def test_batch_launch_collect_protocol(hbe):
    """launch enqueues, collect retires; membership changes wait for collect."""
    r = small_stream(2, 17)
    b = hbe.Batch(hbe.FP32, K=4)
    ss = []
    for q in r:
        s = hbe.Solver(q.N, q.L, q.mu, q.lam, 0, hbe.FP32)
        s.set_initial_bumps(q.bumps)
        ss.append(s)
    b.add(ss[0], 6, 0.01)
    assert b.collect() == []          # nothing in flight
    b.launch()
    with pytest.raises(hbe.HBEError):
        b.add(ss[1], 6, 0.01)         # a run is in flight
    with pytest.raises(hbe.HBEError):
        b.launch()
    assert b.collect() == []          # 4 of 6 steps done
    b.add(ss[1], 6, 0.01)
    done = b.run()
    assert done == [ss[0]]
    assert ss[0].progress()[0] == 6
    b.close()
    for s in ss:
        s.close()
