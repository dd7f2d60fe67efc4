"""Schedule / tile-shape / z-chunk autotuner for the stage kernels.

For a problem size N, boundary kind and precision, both kernel schedules
(four one-stage launches per step, or two fused stage pairs) are run with
every compiled tile variant and a few z-chunk lengths on synthetic data of
that size; the fastest (variant, zchunk, schedule) is kept in a JSON cache
keyed by GPU name, N, boundary and precision.  The cache path is $HBE_AUTOTUNE_CACHE, else
~/.cache/hbe_autotune.json.
"""
from __future__ import annotations

import json
import os
import threading
from typing import Dict, Iterable, Optional, Tuple

import numpy as np

from . import _lib
from .solver import Solver, variants

_lock = threading.Lock()


def cache_path() -> str:
    return os.environ.get("HBE_AUTOTUNE_CACHE",
                          os.path.join(os.path.expanduser("~"), ".cache", "hbe_autotune.json"))


def _gpu_name() -> str:
    import torch
    return torch.cuda.get_device_name()


def _key(N: int, bc: int, prec: int) -> str:
    return f"{_gpu_name()}|N={N}|bc={bc}|prec={_lib.PREC_NAMES[prec]}"


def load_cache() -> Dict[str, dict]:
    path = cache_path()
    if os.path.exists(path):
        try:
            with open(path) as f:
                return json.load(f)
        except (OSError, ValueError):
            return {}
    return {}


def save_cache(cache: Dict[str, dict]) -> None:
    path = cache_path()
    os.makedirs(os.path.dirname(path) or ".", exist_ok=True)
    tmp = path + f".tmp{os.getpid()}"
    with open(tmp, "w") as f:
        json.dump(cache, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def zchunk_candidates(N: int) -> Iterable[int]:
    c = {0, N}
    for d in (2, 3, 4, 6, 8, 12, 16):
        zc = -(-N // d)
        if zc >= 16:
            c.add(zc)
    return sorted(c)


def measure(N: int, bc: int, prec: int, variant: int, zchunk: int, steps: int = 10,
            warmup: int = 3, seed: int = 0, schedule: int = 1) -> float:
    """Seconds per RK4 step of one (variant, zchunk, schedule) on smooth random data."""
    import torch
    rng = np.random.default_rng(seed)
    # smooth data: low Fourier modes only (no stop rule, no special values)
    x = np.linspace(0.0, 2 * np.pi, N, endpoint=False)
    a = rng.uniform(-1, 1, size=3)
    phi0 = (a[0] * np.sin(x)[None, None, :] + a[1] * np.cos(2 * x)[None, :, None]
            + a[2] * np.sin(x + 0.3)[:, None, None]) * np.ones((N, N, N))
    L = 20.0
    h = L / N if bc == _lib.PERIODIC else L / (N + 1)
    with Solver(N, L, 1.0, 1.0, bc, prec) as s:
        s.set_tuning(variant, zchunk)
        s.set_schedule(schedule)
        s.set_initial(torch.from_numpy(phi0).cuda(), torch.zeros((N, N, N), dtype=torch.float64,
                                                                  device="cuda"))
        s.step(warmup, h / 4)
        st = torch.cuda.current_stream()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(st)
        s.step_async(steps, h / 4)
        e1.record(st)
        s.sync()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / 1e3 / steps


def tune(N: int, bc: int, prec: int, steps: int = 10, save: bool = True,
         verbose: bool = False) -> dict:
    """Sweep every schedule x variant x z-chunk; return and cache the fastest."""
    results = []
    for sch in (1, 0):
        for v in range(len(variants(prec))):
            for zc in zchunk_candidates(N):
                t = measure(N, bc, prec, v, zc, steps, schedule=sch)
                results.append((t, v, zc, sch))
                if verbose:
                    print(f"N={N} bc={bc} prec={_lib.PREC_NAMES[prec]} schedule={sch} "
                          f"variant={v} zchunk={zc}: {t * 1e3:.3f} ms/step")
    t, v, zc, sch = min(results)
    entry = {"variant": v, "zchunk": zc, "schedule": sch, "ms_per_step": t * 1e3,
             "gpoint_steps_per_s": N ** 3 / t / 1e9,
             "sweep": [[vv, zz, ss, tt * 1e3] for tt, vv, zz, ss in results]}
    if save:
        with _lock:
            cache = load_cache()
            cache[_key(N, bc, prec)] = entry
            save_cache(cache)
    return entry


def best(N: int, bc: int, prec: int, tune_missing: bool = False) -> Tuple[int, int, int]:
    """(variant, zchunk, schedule) for this size from the cache; (0, 0, 1) =
    the library's default when nothing is cached (or tune now if tune_missing)."""
    cache = load_cache()
    e = cache.get(_key(N, bc, prec))
    if e is None and tune_missing:
        e = tune(N, bc, prec)
    if e is None:
        return 0, 0, 1
    return int(e["variant"]), int(e["zchunk"]), int(e.get("schedule", 1))


def apply(solver: Solver, tune_missing: bool = False) -> Tuple[int, int, int]:
    v, zc, sch = best(solver.N, solver.bc, solver.prec, tune_missing)
    solver.set_tuning(v, zc)
    solver.set_schedule(sch)
    return v, zc, sch


if __name__ == "__main__":
    import argparse
    ap = argparse.ArgumentParser(description="tune the stage kernels for given sizes")
    ap.add_argument("--N", type=int, nargs="+", default=[64, 128, 256, 512])
    ap.add_argument("--bc", type=int, default=_lib.DIRICHLET)
    ap.add_argument("--prec", default="fp32", choices=list(_lib.PREC_NAMES.values()))
    ap.add_argument("--steps", type=int, default=10)
    args = ap.parse_args()
    prec = {v: k for k, v in _lib.PREC_NAMES.items()}[args.prec]
    for n in args.N:
        e = tune(n, args.bc, prec, args.steps, verbose=True)
        print(json.dumps({"N": n, "best": {k: e[k] for k in ("variant", "zchunk", "schedule",
                                                               "ms_per_step",
                                                               "gpoint_steps_per_s")}}))
