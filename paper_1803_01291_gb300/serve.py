"""Continuous-batching server for HBE solve requests.

Requests (an N^3 problem, its parameters, initial data and horizon) arrive
over time.  The server admits each one as soon as a slot and enough device
memory are free, keeps its state on the GPU, and advances every admitted
problem together: one `Batch.run()` replays a CUDA graph of K RK4 steps in
which each stage is a single persistent kernel launch over the tiles of all
members (libhbe's batched runner).  Members leave the batch the moment they
reach their step count (or the stop rule fires), their result is read back,
their memory is released and waiting requests take their place — new work
joins between graph replays without re-capturing the graph.  The next run
is enqueued before the finished members are retired, and their diagnostics
run on a second stream, so the GPU does not wait for the host between runs.

Each member's arithmetic per grid point is the same as when it runs alone,
so results do not depend on what else is in the batch (bitwise).
"""
from __future__ import annotations

import math
import time
from dataclasses import dataclass, field
from typing import Callable, Dict, List, Optional, Sequence

import numpy as np

from . import _lib
from .solver import Batch, Solver, workspace_bytes


@dataclass
class SolveRequest:
    """One problem to solve: N^3 zero-Dirichlet or periodic grid on a box of
    side L, parameters mu, lambda, initial data (host arrays or a callable
    producing them), horizon T and step dt (nsteps = ceil(T/dt - 1e-12))."""
    rid: int
    arrival: float
    N: int
    L: float
    mu: float
    lam: float
    T: float
    dt: float
    init: Optional[Callable[[], tuple]] = None
    bc: int = _lib.DIRICHLET
    # alternative to `init`: phi0 as a sum of bumps (A, R, (cx, cy, cz)), phi1 = 0,
    # evaluated on the device (nothing but the parameters crosses the bus)
    bumps: Optional[Sequence[tuple]] = None

    @property
    def nsteps(self) -> int:
        return int(math.ceil(self.T / self.dt - 1e-12))

    @property
    def work(self) -> float:
        """point-steps of the whole solve"""
        return float(self.N) ** 3 * self.nsteps


@dataclass
class Result:
    rid: int
    arrival: float
    admitted: float
    finished: float
    steps: int
    status: int
    max_abs_phi: float
    phi: Optional[np.ndarray] = None

    @property
    def latency(self) -> float:
        return self.finished - self.arrival


@dataclass
class ServeStats:
    results: List[Result] = field(default_factory=list)
    makespan: float = 0.0
    work: float = 0.0
    runs: int = 0
    peak_members: int = 0
    peak_bytes: int = 0
    launches: int = 0
    admission_retries: int = 0

    def summary(self) -> dict:
        lat = np.array([r.latency for r in self.results]) if self.results else np.zeros(1)
        return {"requests": len(self.results),
                "p50_latency_s": float(np.percentile(lat, 50)),
                "p99_latency_s": float(np.percentile(lat, 99)),
                "mean_latency_s": float(lat.mean()),
                "makespan_s": self.makespan,
                "gpoint_steps_per_s": self.work / self.makespan / 1e9 if self.makespan else 0.0,
                "batch_runs": self.runs, "peak_members": self.peak_members,
                "peak_state_bytes": self.peak_bytes, "gpu_launches": self.launches,
                "admission_retries": self.admission_retries}


class Server:
    """Admission by free device memory and a member cap; continuous batching
    of K-step runs.  `hbm_budget` (bytes) bounds the fields of all members;
    default: 90% of the free device memory at start."""

    def __init__(self, prec: int = _lib.FP32, K: int = 8, hbm_budget: Optional[int] = None,
                 max_members: int = 512, keep_fields: bool = False,
                 tuning: Optional[Callable[[int, int], tuple]] = None):
        import torch
        self.torch = torch
        self.prec = prec
        self.K = K
        if hbm_budget is None:
            free, _ = torch.cuda.mem_get_info()
            hbm_budget = int(0.9 * free)
        self.budget = hbm_budget
        self.max_members = max_members
        self.keep_fields = keep_fields
        self.tuning = tuning
        self.batch = Batch(prec, K)
        self.in_use = 0
        self._live: Dict[int, tuple] = {}
        self._side = None  # stream of the retirement work (diagnostics, reads)
        self._tuned: Dict[tuple, tuple] = {}  # (N, bc) -> (variant, zchunk)

    def need_bytes(self, req: SolveRequest) -> int:
        return workspace_bytes(req.N, req.bc, self.prec)

    def _default_variant(self, N: int) -> int:
        """Tile variant of a member when neither a tuning callback nor the
        autotuner's cache gives one: variant 0 for every size.  One variant
        means one pair of stage launches per step for the whole batch;
        measured on the 256-request stream, that beat giving
        grids below 256^3 the smallest tile (closed-loop capacity 70.1 against
        66.7 Gpoint-steps/s, p99 latency 0.277 against 0.280 s) once the
        stages 1+2 kernels had been made leaner."""
        return 0

    def _cached_tuning(self, N: int, bc: int) -> tuple:
        """(variant, z-chunk) the autotuner recorded for this size, boundary and
        precision (autotune.py's cache), else variant 0 with the automatic
        z-chunk.  Members always run the fused schedule."""
        key = (N, bc)
        if key not in self._tuned:
            try:
                from . import autotune
                e = autotune.load_cache().get(autotune._key(N, bc, self.prec))
            except Exception:
                e = None
            self._tuned[key] = ((int(e["variant"]), int(e["zchunk"])) if e
                                else (self._default_variant(N), 0))
        return self._tuned[key]

    def _out_of_memory(self, e: Exception) -> bool:
        if isinstance(e, _lib.HBEError):
            return e.status == _lib.ENOMEM
        return isinstance(e, getattr(self.torch.cuda, "OutOfMemoryError", ()))

    def _admit(self, req: SolveRequest, now: float):
        torch = self.torch
        s = Solver(req.N, req.L, req.mu, req.lam, req.bc, self.prec)
        if self.tuning is not None:
            v, zc = self.tuning(req.N, self.prec)
        else:
            v, zc = self._cached_tuning(req.N, req.bc)
        s.set_tuning(v, zc)
        if req.bumps is not None:
            s.set_initial_bumps(req.bumps)
        else:
            phi0, phi1 = req.init()
            s.set_initial(torch.from_numpy(np.ascontiguousarray(phi0)).cuda(),
                          torch.from_numpy(np.ascontiguousarray(phi1)).cuda())
        self.batch.add(s, req.nsteps, req.dt)
        nb = self.need_bytes(req)
        self.in_use += nb
        self._live[s.handle.value] = (req, s, now, nb)

    def run(self, requests: Sequence[SolveRequest], clock: Callable[[], float] = time.perf_counter,
            realtime: bool = True) -> ServeStats:
        """Serve the requests (sorted by arrival).  realtime=True honours the
        arrival times against `clock`; False admits as if every request had
        already arrived (closed-loop capacity run)."""
        pending = sorted(requests, key=lambda r: r.arrival)
        for r in pending:
            if self.need_bytes(r) > self.budget:
                raise ValueError(f"request {r.rid} (N={r.N}) needs more than the whole budget")
        stats = ServeStats()
        t0 = clock()
        i = 0
        in_flight = False
        while i < len(pending) or len(self.batch) or in_flight:
            # the run in flight: wait for it, take its finished members out
            done = []
            if in_flight:
                done = self.batch.collect()
                in_flight = False
            now = clock() - t0
            # admission: arrived, fits in memory, slot free (FIFO, no overtaking)
            while i < len(pending):
                r = pending[i]
                if realtime and r.arrival > now:
                    break
                nb = self.need_bytes(r)
                if self.in_use + nb > self.budget or len(self.batch) >= self.max_members:
                    break
                try:
                    self._admit(r, now)
                except Exception as e:  # out of device memory: wait for a member to leave
                    if not self._out_of_memory(e) or not len(self.batch):
                        raise
                    stats.admission_retries += 1
                    break
                stats.work += r.work
                i += 1
            stats.peak_members = max(stats.peak_members, len(self.batch))
            stats.peak_bytes = max(stats.peak_bytes, self.in_use)
            # the next run goes to the GPU before the finished members are
            # retired, so their diagnostics and reads overlap it
            if len(self.batch):
                l0 = self.batch.launches
                self.batch.launch()
                in_flight = True
                stats.launches += self.batch.launches - l0
                stats.runs += 1
            self._retire(done, stats, t0, clock, realtime)
            if not in_flight and not done and i < len(pending):
                wait = pending[i].arrival - (clock() - t0)
                if wait > 0:
                    time.sleep(min(wait, 0.05))
        stats.makespan = clock() - t0
        return stats

    def _retire(self, done, stats: ServeStats, t0: float, clock, realtime: bool):
        """Results of the members that left the batch: status, step count, the
        diagnostics (max|phi|, bubble count) and optionally phi, computed on a
        side stream while the batch's next run occupies the main one."""
        if not done:
            return
        torch = self.torch
        if self._side is None and torch.cuda.is_available():
            self._side = torch.cuda.Stream()
        for s in done:
            req, _, admitted, nb = self._live.pop(s.handle.value)
            st = s.sync()
            steps, _ = s.progress()
            if self._side is not None:
                s.set_stream(self._side.cuda_stream)
            d = s.diag()  # the result: max|phi|, finiteness, bubble count
            phi = s.read(psi=False)[0] if self.keep_fields else None
            # closed-loop runs treat every request as arrived at the start
            arrived = req.arrival if realtime else 0.0
            stats.results.append(Result(req.rid, arrived, admitted, clock() - t0, steps,
                                        st, d["max_abs_phi"], phi))
            s.close()
            self.in_use -= nb

    def close(self):
        self.batch.close()


def requests_from_stream(stream, device_init: bool = True) -> List[SolveRequest]:
    """SolveRequests from seeded request records (N, L, mu, lam, T, bumps,
    arrival, rid, and steps() -> (nsteps, dt <= h/4)); the initial data is
    built on the device from the bump parameters unless device_init is False."""
    out = []
    for r in stream:
        n, dt = r.steps()
        out.append(SolveRequest(r.rid, r.arrival, r.N, r.L, r.mu, r.lam, r.T, dt,
                                init=None if device_init else r.initial,
                                bumps=list(r.bumps) if device_init else None))
    return out


def run_alone(requests: Sequence[SolveRequest], prec: int = _lib.FP64) -> dict:
    """Each request solved by itself, one after another (no batching), in the
    given precision: the baseline the batched server is compared with."""
    import torch
    t0 = time.perf_counter()
    lat, work = [], 0.0
    for r in sorted(requests, key=lambda q: q.arrival):
        ts = time.perf_counter()
        with Solver(r.N, r.L, r.mu, r.lam, r.bc, prec) as s:
            if r.bumps is not None:
                s.set_initial_bumps(r.bumps)
            else:
                a, b = r.init()
                s.set_initial(a, b)
            s.step(r.nsteps, r.dt)
            s.diag()
        lat.append(time.perf_counter() - ts)
        work += r.work
    total = time.perf_counter() - t0
    lat = np.array(lat)
    return {"requests": len(lat), "total_s": total, "gpoint_steps_per_s": work / total / 1e9,
            "p50_solve_s": float(np.percentile(lat, 50)),
            "p99_solve_s": float(np.percentile(lat, 99))}
