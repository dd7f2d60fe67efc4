"""Throughput benchmark of the HBE RK4 + FD4 hot path on GB300.

Workload: 512^3 unknowns on the periodic box [-20, 20]^3, mu = 1, lambda = 1,
phi0 = seeded band-limited Gaussian random field (std 1, correlation length 2,
seed 0), phi1 = 0, dt = T/nsteps <= h/4 (T = 6, 308 steps), FP32 fields with
compensated (hi, lo) phi/psi and FP64 time/e^{-2t} coefficients.  One bench
step = one full RK4 step (all four stage kernels) over the whole grid.

Metric: Gpoint-steps/s = N^3 x steps / seconds (whole job: summed over ranks).
The FP64, BF16-storage and plain-FP32 paths are measured on the same GPU and
reported beside it.  The field state (>= 4 x 512 MiB) is larger than L2, so
no flush is needed between steps.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

With --impl reference the CPU oracle (plain FP64 C, all host cores) is timed
on the same workload, each step one RK4 step on a 512 x 512 x 64 slab of it.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N_DEFAULT = 512
L_BOX = 40.0
HORIZON = 6.0

# algorithmic bytes per point of each stage kernel (reads + writes of the fields
# a stage touches once each), per precision: (state bytes, G bytes, compensated)
PREC_BYTES = {"fp64": (8, 8, False), "fp32": (4, 4, True), "bf16": (4, 2, True),
              "fp32_plain": (4, 4, False)}


def stage_bytes(prec: str, schedule: int = 1):
    """Algorithmic bytes per grid point of each launch of one RK4 step."""
    s, g, comp = PREC_BYTES[prec]
    lo = 4 * s if comp else 0      # lo parts of p and q, in and out
    if schedule == 1:
        a = 2 * s + 2 * g          # p, q -> G1, G2
        b = 2 * s + 2 * g + 2 * s + lo  # p, q, G1, G2 -> p', q'
        return [a, b]
    b1 = 2 * s + g                 # p, q -> G1
    b2 = 2 * s + 2 * g             # p, q, G1 -> G2
    b3 = 2 * s + 3 * g             # p, q, G1, G2 -> G3
    b4 = 2 * s + 3 * g + 2 * s + lo  # p, q, G1, G2, G3 -> p', q'
    return [b1, b2, b3, b4]


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return d.get("hbm_gbs", 6800.0), "measured"
    return 6800.0, "fallback"


# FP64 FMA rate of GB300 measured with a dependent-free FMA loop (0.58 TFMA/s,
# 152 SMs, ~1.9 GHz): the FP64 stage kernels are bound by it, not by HBM.
FP64_FMA_PER_S = 0.58e12
# FP64 instructions (DADD + DFMA + DMUL) per point-step of the fused FP64
# kernels, counted by ncu on the 256^3 periodic workload (38.3 + 61.0)
FP64_INSTR_PER_POINT_STEP = 99.3


def kernel_source_hash(prec: str = "fp32") -> str:
    """Hash of the stage-kernel sources and the precision's tile-variant table."""
    h = hashlib.sha256()
    for fn in ("hbe_stage.cuh", "hbe_common.cuh", f"hbe_stage_{prec}.cu"):
        with open(os.path.join(ROOT, "paper_1803_01291_gb300", "csrc", fn), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def tuned(hbe, N: int, bc: int, prec: int):
    """(variant, zchunk, schedule) from the autotuner cache if present, else
    the library's defaults."""
    from paper_1803_01291_gb300 import autotune
    try:
        return autotune.best(N, bc, prec)
    except Exception:
        return (0, 0, 1)


def recorded_traffic(prec: str, N: int, schedule: int = 1):
    """dram bytes per launch of the dominant kernel from the committed ncu summary,
    if it was taken on the current kernel source."""
    kind = "pair34" if schedule == 1 else "stage4"
    path = os.path.join(ROOT, "profiles", f"{kind}_{prec}_traffic.txt")
    if not os.path.exists(path):
        return None
    kv = {}
    for line in open(path):
        if "=" in line and not line.startswith("#"):
            k, v = line.split("=", 1)
            kv[k.strip()] = v.strip()
    if kv.get("kernel_source_sha256_16") != kernel_source_hash(prec):
        return None
    try:
        per_point = float(kv["dram_bytes_per_point"])
    except (KeyError, ValueError):
        return None
    return per_point * N ** 3


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.QUERY}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self._t = threading.Thread(target=self._read, daemon=True)
            self._t.start()
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self._t.join(timeout=2)

    def summary(self):
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = float(parts[2])
            except ValueError:
                continue
            for name, val in zip(names, parts[5:9]):
                if val.lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_setup(gpus: int):
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world != gpus and world != 1:
        raise SystemExit(f"--gpus {gpus} but WORLD_SIZE={world}")
    # torchrun sets the rendezvous; a bare run is rank 0 of 1
    return rank, world, local


def barrier(world, torch):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(value: float, world, torch, device):
    if world == 1:
        return value
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate(units_per_rank: float, secs_max: float, world: int) -> float:
    """Whole-job throughput in units of 1e9 per second: every rank's units over
    the slowest rank's time (weak scaling: each rank solves its own replica)."""
    return units_per_rank * world / secs_max / 1e9


def workload(N: int):
    import hbe_inputs as hi
    prob = hi.grf_problem(N, lam=1.0, seed=0)
    return prob


def time_path(hbe, torch, prob, prec_id, steps, warmup, schedule=1, tuning=None):
    """Warm up, then time `steps` RK4 steps through the production path (the
    context's CUDA graph of K steps, hbe_step_async) with CUDA events on the
    solver's stream.  The per-kernel times for the roofline come from a
    separate run with every kernel bracketed by events (hbe_profile_stages).
    Returns (seconds, per-launch ms, launches in the timed region)."""
    s = hbe.Solver(prob.N, prob.L, prob.mu, prob.lam, prob.bc, prec_id)
    s.set_schedule(schedule)
    if tuning is not None:
        s.set_tuning(tuning[0], tuning[1])
    phi0 = torch.from_numpy(prob.phi0).cuda()
    phi1 = torch.from_numpy(prob.phi1).cuda()
    s.set_initial(phi0, phi1)
    del phi0, phi1
    if warmup:
        s.step(warmup, prob.dt)  # also captures the graph
    stage_ms = s.profile_stages(min(steps, 50), prob.dt)
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    l0 = s.launches
    e0.record(stream)
    s.step_async(steps, prob.dt)
    e1.record(stream)
    s.sync()
    torch.cuda.synchronize()
    secs = e0.elapsed_time(e1) / 1e3
    # the library's count (stage and ghost-copy kernels of every graph replay,
    # K steps each) + two bookkeeping kernels per replay (step coefficients,
    # advance) + one run-setup kernel
    K = 8
    launches = s.launches - l0 + 2 * ((steps + K - 1) // K) + 1
    s.close()
    return secs, stage_ms, launches


def e2e_buffers(torch, prob):
    """Pinned host buffers of one solve (phi0, phi1 in, phi out), allocated at
    the start of the run, before the other legs allocate and free host memory
    (copies from buffers pinned after them were at times 8x slower)."""
    N = prob.N
    h0 = torch.from_numpy(prob.phi0).pin_memory()
    h1 = torch.from_numpy(prob.phi1).pin_memory()
    out = torch.empty((N, N, N), dtype=torch.float64).pin_memory()
    return h0, h1, out


def e2e_solve(hbe, torch, prob, prec_id, nsteps, solves=3, buffers=None):
    """`solves` back-to-back solves through the public API with host buffers:
    initial data from pinned host memory, nsteps on the GPU, phi back to
    pinned host memory.  Returns the total time and the phases of each solve."""
    import numpy as np
    import ctypes
    N = prob.N
    h0, h1, out = buffers if buffers is not None else e2e_buffers(torch, prob)
    s = hbe.Solver(N, prob.L, prob.mu, prob.lam, prob.bc, prec_id)
    tt = ctypes.c_double()
    dp = ctypes.POINTER(ctypes.c_double)
    # warm (graph capture, staging buffers, both copy directions)
    s.set_initial(h0.numpy(), h1.numpy())
    s.step(2, prob.dt)
    s.lib.hbe_read(s.handle, ctypes.cast(out.data_ptr(), dp), None, ctypes.byref(tt))
    torch.cuda.synchronize()
    phases, st = [], 0
    t_start = time.perf_counter()
    for _ in range(solves):
        t0 = time.perf_counter()
        s.set_initial(h0.numpy(), h1.numpy())
        t1 = time.perf_counter()
        st = s.step(nsteps, prob.dt)
        t2 = time.perf_counter()
        s.lib.hbe_read(s.handle, ctypes.cast(out.data_ptr(), dp), None, ctypes.byref(tt))
        t3 = time.perf_counter()
        phases.append({"initial_data_s": t1 - t0, "steps_s": t2 - t1, "read_s": t3 - t2})
    total = time.perf_counter() - t_start
    s.close()
    return total, st, float(np.abs(out.numpy()).max()), phases


def e2e_solve_pipelined(hbe, torch, prob, prec_id, nsteps, solves=5, buffers=None):
    """`solves` back-to-back solves through the C ABI with host buffers, as a
    user streaming problems through one context runs them: while solve k
    steps, solve k+1's phi0, phi1 are prefetched from pinned host memory
    (`hbe_prefetch_initial`, DMA on the context's copy stream) and solve k-1's
    phi, read with `hbe_read_async`, crosses back to pinned host memory the
    same way.  The first solve's inputs and the last solve's phi, which nothing
    overlaps, take the direct path (the pack / unpack kernels read and write
    the pinned host arrays).  Every copy is inside the timed region.  Returns
    the total time and the critical-path phases of each solve."""
    import numpy as np
    import ctypes
    N = prob.N
    h0, h1, out = buffers if buffers is not None else e2e_buffers(torch, prob)
    a0, a1, o = h0.numpy(), h1.numpy(), out.numpy()
    s = hbe.Solver(N, prob.L, prob.mu, prob.lam, prob.bc, prec_id)
    tt = ctypes.c_double()
    dp = ctypes.POINTER(ctypes.c_double)

    def read_direct():
        s.lib.hbe_read(s.handle, ctypes.cast(out.data_ptr(), dp), None, ctypes.byref(tt))

    # warm (graph capture, staging areas, both paths and directions)
    s.prefetch_initial(a0, a1)
    s.set_initial_prefetched()
    s.step(2, prob.dt)
    s.read_async(o)
    s.read_wait()
    s.set_initial(a0, a1)
    read_direct()
    torch.cuda.synchronize()
    phases, st = [], 0
    t_start = time.perf_counter()
    for k in range(solves):
        t0 = time.perf_counter()
        if k == 0:
            s.set_initial(a0, a1)
        else:
            s.set_initial_prefetched()
        t1 = time.perf_counter()
        s.step_async(nsteps, prob.dt)
        if k + 1 < solves:
            s.prefetch_initial(a0, a1)   # overlaps this solve's steps
        st = s.sync()
        t2 = time.perf_counter()
        if k + 1 < solves:
            s.read_async(o)              # its copy overlaps the next solve
        else:
            s.read_wait()
            read_direct()
        t3 = time.perf_counter()
        phases.append({"initial_data_s": t1 - t0, "steps_s": t2 - t1, "read_s": t3 - t2})
    total = time.perf_counter() - t_start
    s.close()
    return total, st, float(np.abs(o).max()), phases


def serve_leg(hbe, count: int = 256, seed: int = 0, load: float = 0.8):
    """Continuous batching on the seeded stream of `count` solve requests
    (N in {32..256}^3, mu, lambda ~ U[.5, 2], 1-4 bumps, T ~ U[1, 6], FP32 with
    compensated state).  A closed-loop run measures the batched capacity; the
    Poisson arrival rate is then set to `load` x capacity and the stream is
    served in real time (p50/p99 latency = finish - arrival).  Baseline: the
    same requests solved one after another, alone, on the FP64 path."""
    import hbe_inputs as hi
    from paper_1803_01291_gb300 import serve
    stream = hi.request_stream(count, seed=seed, rate=1.0)
    reqs = serve.requests_from_stream(stream)
    total = sum(r.work for r in reqs)
    srv = serve.Server(hbe.FP32, K=8)
    cal = srv.run(reqs, realtime=False)
    srv.close()
    capacity = total / cal.makespan                  # point-steps / s
    rate = load * capacity / (total / count)         # requests / s
    for r in reqs:
        r.arrival = r.arrival / rate                 # the stream was drawn at rate 1
    srv = serve.Server(hbe.FP32, K=8)
    live = srv.run(reqs, realtime=True)
    srv.close()
    alone = serve.run_alone(reqs, hbe.FP64)
    out = live.summary()
    out.update({"closed_loop_gpoint_steps_per_s": capacity / 1e9,
                "arrival_rate_req_per_s": rate, "load": load,
                "alone_fp64": alone,
                "speedup_vs_alone_fp64": out["gpoint_steps_per_s"] / alone["gpoint_steps_per_s"],
                "workload": f"{count} requests, seed {seed}, N in {{32,48,64,96,128,192,256}}^3, "
                            "zero-Dirichlet [-10,10]^3, FP32 compensated, K = 8 steps per graph"})
    return out


def cpu_baseline(prob, nsteps=2):
    """The oracle as it stands, on all host cores, nsteps RK4 steps of the full grid."""
    import oracle
    cores = os.cpu_count() or 1
    t0 = time.perf_counter()
    oracle.run(prob.phi0, prob.phi1, prob.L, prob.mu, prob.lam, prob.bc, 0.0, prob.dt, nsteps,
               nthreads=cores)
    secs = time.perf_counter() - t0
    pts = prob.N ** 3 * nsteps
    return {"value": pts / secs / 1e9, "unit": "Gpoint-steps/s", "cores": cores, "kind": "oracle",
            "sample": f"{nsteps} RK4 steps of the full {prob.N}^3 workload (FP64 C oracle, "
                      f"OpenMP over z, {cores} threads), {secs:.2f} s"}


# floating-point operations of one radial node-step (four stages of the Laplacian
# with its 2/r term, 14; the right-hand side, 9; the stage arguments and the RK4
# combine), counted with an FMA as two
RADIAL_FLOPS_PER_NODE_STEP = 121
# FP32 lanes: 152 SMs x 128 lanes x 2 flops (FMA) x 2.07 GHz
FP32_PEAK_FLOPS = 152 * 128 * 2 * 2.07e9


def radial_workload(batch: int = 1216, n: int = 2000, seed: int = 0):
    """A seeded parameter sweep of radial problems in the paper's units (Sec. 3:
    L = 5, the bump B(r; 0, R0), mu^2 in [0.1, 9], lambda in [0.1, 2]): phi0 =
    A B(r; 0, R0) with A in [0.5, 3], R0 in [0.1, 0.4] (unit box), phi1 = kappa
    phi0 with kappa in [-5, 5]; n nodes on [0, 5], dt = 1e-3, 2000 steps."""
    import numpy as np
    rng = np.random.default_rng(seed)
    R = 5.0
    r = np.arange(n) * R / n / R  # unit-box radius
    A = rng.uniform(0.5, 3.0, batch)
    R0 = rng.uniform(0.1, 0.4, batch)
    kap = rng.uniform(-5.0, 5.0, batch)
    mu = np.sqrt(rng.uniform(0.1, 9.0, batch))
    lam = rng.uniform(0.1, 2.0, batch)
    s = (r[None, :] / R0[:, None]) ** 2
    inside = s < 1
    B = np.zeros((batch, n))
    B[inside] = np.exp((1.0 / R0[:, None] ** 2 - 1.0 / (R0[:, None] ** 2 - r[None, :] ** 2))[inside])
    phi0 = A[:, None] * B
    phi1 = kap[:, None] * phi0
    dt = R / n / 4
    return {"R": R, "n": n, "dt": dt, "nsteps": int(round(2.0 / dt)), "phi0": phi0, "phi1": phi1,
            "mu": mu, "lam": lam}


def radial_leg(hbe, torch, cpu: bool = True):
    """Batched radial solver (Sec. 2.2) on the sweep above, FP32 and FP64:
    node-steps per second over one launch that integrates every problem, timed
    with CUDA events; the FP32 roofline is the FP32 FMA rate of the SMs, the
    FP64 one the measured FP64 FMA rate.  CPU: the radial oracle (FP64 numpy)
    on one problem for 20000 steps."""
    from paper_1803_01291_gb300 import radial
    w = radial_workload()
    B, n = w["phi0"].shape
    phi0 = torch.from_numpy(w["phi0"]).cuda()
    phi1 = torch.from_numpy(w["phi1"]).cuda()
    out = {"workload": f"{B} radial problems, n = {n} nodes on [0, 5], dt = {w['dt']:g}, "
                       f"{w['nsteps']} steps, records every 100 steps, stop at 1e6 (seed 0)"}
    for name, prec, peak in (("fp32", hbe.FP32, FP32_PEAK_FLOPS),
                             ("fp64", hbe.FP64, 2 * FP64_FMA_PER_S)):
        radial.run(phi0, phi1, w["R"], w["mu"], w["lam"], 0.0, w["dt"], 20, prec=prec)
        stream = torch.cuda.current_stream()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        res = radial.run(phi0, phi1, w["R"], w["mu"], w["lam"], 0.0, w["dt"], w["nsteps"],
                         prec=prec, record_every=100, stop=1e6)
        e1.record(stream)
        torch.cuda.synchronize()
        secs = e0.elapsed_time(e1) / 1e3
        node_steps = float(res.steps.sum().item()) * n
        rate = node_steps / secs
        out[name] = {"value": rate / 1e9, "unit": "Gnode-steps/s", "seconds": secs,
                     "stopped": int((res.status.cpu() != 0).sum().item()),
                     "roofline": {"bound": "alu", "achieved": rate * RADIAL_FLOPS_PER_NODE_STEP / 1e12,
                                  "peak": peak / 1e12, "unit": "TFLOP/s",
                                  "frac": rate * RADIAL_FLOPS_PER_NODE_STEP / peak,
                                  "peak_kind": "nominal FP32 FMA rate (152 SMs x 128 lanes x 2.07 GHz)"
                                  if prec == hbe.FP32 else "measured FP64 FMA rate"}}
    if cpu:
        import oracle.radial_phi as rp
        t0 = time.perf_counter()
        rp.run(w["phi0"][0], w["phi1"][0], w["R"], w["mu"][0], w["lam"][0], 0.0, w["dt"], 20000)
        secs = time.perf_counter() - t0
        out["cpu_baseline"] = {"value": n * 20000 / secs / 1e9, "unit": "Gnode-steps/s",
                               "cores": 1, "kind": "oracle",
                               "sample": f"one problem of the sweep, 20000 steps (FP64 numpy, one "
                                         f"core), {secs:.2f} s"}
    return out


METRIC = "Gpoint-steps/s at 512^3 (FP32 vs FP64, same GB300); p50/p99 serve latency"


def workload_config(N, prob, world=1):
    return {"workload": "hbe-512-periodic-grf", "N": N, "L": L_BOX, "mu": 1.0, "lambda": 1.0,
            "bc": "periodic", "seed": 0, "dt": prob.dt,
            "precision": "fp32 fields and math, compensated phi/psi, fp64 t and e^{-2t}",
            "l2": "state > L2 (4 x 512 MiB fields), no flush needed",
            "parallelism": f"replicas x{world}" if world > 1 else "single GPU"}


def reference_arm(args):
    """CPU oracle timed as the reference implementation (rank 0 only).  Each
    bench step is one RK4 step of the oracle on a 512 x 512 x S slab of the
    workload (periodic), S chosen once from a probe step so that the whole run
    stays near two minutes."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import numpy as np
    import oracle
    N = args.N
    prob = workload(N)
    h = prob.L / N
    cores = os.cpu_count() or 1

    def one(slab):
        w0 = np.ascontiguousarray(prob.phi0[:slab])
        w1 = np.ascontiguousarray(prob.phi1[:slab])
        t0 = time.perf_counter()
        oracle.run_box(w0, w1, h, prob.mu, prob.lam, 1, 0.0, prob.dt, 1, nthreads=cores)
        return time.perf_counter() - t0

    probe = one(16)
    budget = 120.0 / (args.steps + args.warmup)
    slab = int(max(4, min(64, 16 * budget / max(probe, 1e-6))) // 4 * 4)
    for _ in range(args.warmup):
        one(slab)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        one(slab)
    secs = time.perf_counter() - t0
    val = N * N * slab * args.steps / secs / 1e9
    sample = f"each step: 1 RK4 step of the FP64 C oracle on a {N}x{N}x{slab} slab ({cores} threads)"
    cfg = workload_config(N, prob)
    cfg["sample"] = sample
    line = {
        "impl": "reference", "metric": METRIC, "value": val, "unit": "Gpoint-steps/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": secs / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": cfg,
        "cpu_baseline": {"value": val, "unit": "Gpoint-steps/s", "cores": cores, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": val, "unit": "Gpoint-steps/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=300)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--N", type=int, default=N_DEFAULT)
    ap.add_argument("--no-extra", action="store_true", help="skip FP64/BF16/plain legs")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU-baseline leg")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-serve", action="store_true", help="skip the serving leg")
    ap.add_argument("--serve-requests", type=int, default=256)
    ap.add_argument("--no-radial", action="store_true", help="skip the batched radial leg")
    ap.add_argument("--schedule", type=int, default=None, choices=[0, 1],
                    help="0: one kernel per RK stage, 1: two fused stage pairs per step "
                         "(default: the autotuner's choice, else 1)")
    args = ap.parse_args()
    if args.warmup < 3:
        raise SystemExit("--warmup must be >= 3")
    if args.impl == "reference":
        reference_arm(args)
        return

    import torch
    rank, world, local = dist_setup(args.gpus)
    torch.cuda.set_device(local)
    device = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=device)
    import paper_1803_01291_gb300 as hbe

    N = args.N
    prob = workload(N)
    e2e_bufs = None if args.no_e2e else e2e_buffers(torch, prob)
    hbm_peak, peak_kind = measured_peaks()

    # headline: FP32 with compensated state; each rank solves its own replica
    tuning = tuned(hbe, N, prob.bc, hbe.FP32)
    if args.schedule is None:
        args.schedule = tuning[2]
    barrier(world, torch)
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        secs, stage_ms, launches = time_path(hbe, torch, prob, hbe.FP32, args.steps, args.warmup,
                                             args.schedule, tuning)
    secs = max_over_ranks(secs, world, torch, device)
    barrier(world, torch)
    value = aggregate(float(N) ** 3 * args.steps, secs, world)

    sb = stage_bytes("fp32", args.schedule)
    nl = len(sb)
    stage_gbs = [sb[i] * N ** 3 / (stage_ms[i] / 1e3) / 1e9 for i in range(nl)]
    dom = max(range(nl), key=lambda i: stage_ms[i])   # the dominant kernel
    names = (["stages 1+2", "stages 3+4 + RK4 combine"] if args.schedule == 1 else
             ["stage 1", "stage 2", "stage 3", "stage 4 + RK4 combine"])
    traffic = recorded_traffic("fp32", N, args.schedule)
    step_gbs = sum(sb) * N ** 3 * args.steps / secs / 1e9
    roofline = {"bound": "hbm", "kernel": f"stage_kernel<FP32> {names[dom]}",
                "achieved": stage_gbs[dom], "peak": hbm_peak, "unit": "GB/s",
                "frac": stage_gbs[dom] / hbm_peak, "peak_kind": peak_kind,
                "traffic": traffic,
                "algorithmic_bytes_per_launch": sb[dom] * N ** 3,
                "step": {"bytes_per_point": sum(sb), "achieved_gbs": step_gbs,
                         "frac": step_gbs / hbm_peak},
                "launches": [{"kernel": names[i], "ms": stage_ms[i], "bytes_per_point": sb[i],
                              "gbs": stage_gbs[i], "frac": stage_gbs[i] / hbm_peak}
                             for i in range(nl)],
                "schedule": args.schedule, "tuning": {"variant": tuning[0], "zchunk": tuning[1]}}

    line = {
        "metric": METRIC,
        "value": value, "unit": "Gpoint-steps/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": secs / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": workload_config(N, prob, world),
        "roofline": roofline,
        "clocks": clk.summary(),
        "gpu_launches": launches,
    }

    # end to end right after the headline leg, before the other precisions' legs
    if not args.no_e2e:
        nsteps = 308 if N == 512 else max(8, int(round(HORIZON / prob.dt)))
        solves, seq_solves = 5, 3
        e2e_secs, st, _, phases = e2e_solve_pipelined(hbe, torch, prob, hbe.FP32, nsteps,
                                                      solves, e2e_bufs)
        seq_secs, _, _, seq_phases = e2e_solve(hbe, torch, prob, hbe.FP32, nsteps, seq_solves,
                                               e2e_bufs)
        e2e_bufs = None
        e2e_secs = max_over_ranks(e2e_secs, world, torch, device)
        seq_secs = max_over_ranks(seq_secs, world, torch, device)
        line["e2e"] = {"value": float(N) ** 3 * nsteps * solves * world / e2e_secs / 1e9,
                       "unit": "Gpoint-steps/s",
                       "h2d_bytes_per_step": 2 * 8 * N ** 3 / nsteps,
                       "d2h_bytes_per_step": 8 * N ** 3 / nsteps,
                       "steps_per_solve": nsteps, "solves": solves,
                       "phases": phases,
                       "note": "back-to-back solves through one context and the C ABI with "
                               "pinned host buffers, each: phi0, phi1 in, nsteps RK4 steps, phi "
                               "out; the next solve's inputs (hbe_prefetch_initial) and the "
                               "previous solve's phi (hbe_read_async) cross the host link by DMA "
                               "while a solve steps, the first inputs and the last phi on the "
                               "direct path; bytes amortised per RK4 step",
                       "sequential": {
                           "value": float(N) ** 3 * nsteps * seq_solves * world / seq_secs / 1e9,
                           "solves": seq_solves, "phases": seq_phases,
                           "note": "each solve's copies on its own critical path (pack / unpack "
                                   "kernels reading and writing the pinned host arrays)"}}

    if not args.no_extra:
        extra = {}
        for name, pid, steps in (("fp64", hbe.FP64, max(10, min(100, args.steps))),
                                 ("bf16", hbe.BF16, args.steps),
                                 ("fp32_plain", hbe.FP32_PLAIN, args.steps)):
            s2, ms2, _ = time_path(hbe, torch, prob, pid, steps, 3, args.schedule,
                                   tuned(hbe, N, prob.bc, pid))
            sbp = stage_bytes(name, args.schedule)
            v = float(N) ** 3 * steps / s2 / 1e9
            entry = {"value": v, "unit": "Gpoint-steps/s", "steps": steps,
                     "ms_per_step": s2 / steps * 1e3, "stage_ms": ms2,
                     "hbm_frac": sum(sbp) * float(N) ** 3 * steps / s2 / 1e9 / hbm_peak}
            if name == "fp64":
                # FP64-pipe roofline: FP64 instructions per point-step of the two fused
                # kernels (ncu count) against the measured FP64 instruction rate
                ach = FP64_INSTR_PER_POINT_STEP * v * 1e9
                entry["roofline"] = {"bound": "alu", "pipe": "fp64", "achieved": ach / 1e12,
                                     "peak": FP64_FMA_PER_S / 1e12, "unit": "T FP64 instr/s",
                                     "frac": ach / FP64_FMA_PER_S,
                                     "per_point_step": FP64_INSTR_PER_POINT_STEP}
            extra[name] = entry
        line["precisions"] = extra

    if not args.no_serve:
        line["serve"] = serve_leg(hbe, args.serve_requests)

    if not args.no_radial:
        line["radial"] = radial_leg(hbe, torch, cpu=(rank == 0 and not args.no_cpu))

    if rank == 0 and world == 1 and not args.no_cpu:
        line["cpu_baseline"] = cpu_baseline(prob, 6 if N >= 512 else 2)

    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
