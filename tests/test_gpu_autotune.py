"""Autotuner: sweeps every tile variant x z-chunk candidate, caches the fastest,
and a tuned solver computes the same bits as the default one."""
import json
import os

import numpy as np
import pytest

import __graft_entry__  # noqa: F401

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hbe():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_1803_01291_gb300 as m
    return m


def test_tune_caches_and_applies(hbe, tmp_path, monkeypatch):
    from paper_1803_01291_gb300 import autotune
    monkeypatch.setenv("HBE_AUTOTUNE_CACHE", str(tmp_path / "cache.json"))
    N = 48
    entry = autotune.tune(N, 0, hbe.FP32, steps=3)
    nvar = len(hbe.variants(hbe.FP32))
    assert len(entry["sweep"]) == 2 * nvar * len(list(autotune.zchunk_candidates(N)))
    best = min(entry["sweep"], key=lambda r: r[3])
    assert (entry["variant"], entry["zchunk"], entry["schedule"]) == tuple(best[:3])
    cache = json.load(open(tmp_path / "cache.json"))
    assert len(cache) == 1
    assert autotune.best(N, 0, hbe.FP32) == (entry["variant"], entry["zchunk"], entry["schedule"])
    rng = np.random.default_rng(1)
    phi0 = rng.standard_normal((N, N, N)) * 0.1
    out = []
    for tuned in (False, True):
        with hbe.Solver(N, 10.0, 1.0, 1.0, 0, hbe.FP32) as s:
            if tuned:
                autotune.apply(s)
            s.set_initial(phi0, np.zeros_like(phi0))
            s.step(4, 10.0 / 49 / 4)
            out.append(s.read()[0])
    assert np.array_equal(out[0], out[1])
