"""The computational examples of Sec. 3 of the paper, run with this solver.

The paper solves the rescaled problem on the unit box [0, 1]^3 with the factor
1/L^2, L = 5, n = 500 intervals per axis (499 unknowns), delta t = 1e-4, and
initial data built from its bump B(x; C, R) (Eq. bump, peak 1).  Here the same
problem is the box of side L = 5 centred at the origin (unit coordinate
u = x / L + 1/2), N = 499 unknowns, zero-Dirichlet boundary, and by default
dt = 1e-3 (the paper's 1e-4 is far inside the stability bound; the
figure-level behaviour is the same).  Each example reports what the paper
reads off its figures: signs, extrema, the bubble count, the integral of phi
and the Laplacian monitor P(t), plus line profiles along the x mid-line and
the main diagonal (the two lines the paper plots).

Run:  python -m paper_1803_01291_gb300.paper_examples [--out DIR] [--n 500] [--dt 1e-3]
"""
from __future__ import annotations

import argparse
import json
import math
import os
import time
from dataclasses import dataclass, field
from typing import Callable, Dict, List, Sequence, Tuple

import numpy as np

from . import _lib
from .solver import Solver

L_PAPER = 5.0


def unit_coords(N: int) -> np.ndarray:
    """Unit-box coordinate of the Dirichlet nodes (i + 1) / (N + 1)."""
    return (np.arange(N) + 1.0) / (N + 1)


def bump_B(N: int, C: Sequence[float], R: float) -> np.ndarray:
    """B(x; C, R) = exp(1/R^2 - 1/(R^2 - |x - C|^2)) inside the ball, else 0
    (Eq. bump), sampled at the unit-box nodes, array [z, y, x]."""
    u = unit_coords(N)
    out = np.zeros((N, N, N))
    sl = []
    for c in (C[2], C[1], C[0]):
        idx = np.nonzero(np.abs(u - c) < R)[0]
        if idx.size == 0:
            return out
        sl.append(slice(int(idx[0]), int(idx[-1]) + 1))
    dz = (u[sl[0]] - C[2])[:, None, None]
    dy = (u[sl[1]] - C[1])[None, :, None]
    dx = (u[sl[2]] - C[0])[None, None, :]
    r2 = dx * dx + dy * dy + dz * dz
    sub = np.zeros_like(r2)
    inside = r2 < R * R
    sub[inside] = np.exp(1.0 / (R * R) - 1.0 / (R * R - r2[inside]))
    out[tuple(sl)] = sub
    return out


@dataclass
class Example:
    name: str
    mu2: float
    lam: float
    init: Callable[[int], Tuple[np.ndarray, np.ndarray]]
    times: List[float]
    line: str = "mid"  # "mid" (x mid-line) or "diag" (main diagonal)
    stop: float = 0.0
    notes: str = ""


MID = (0.5, 0.5, 0.5)


def _ex2(N):
    b = bump_B(N, MID, 0.2)
    return 2 * b, 10 * b


def _ex3(N):
    b = bump_B(N, MID, 0.3)
    return b, -5 * b


def _ex5(N):
    return 3 * bump_B(N, MID, 0.3), np.zeros((N, N, N))


def _ex6(N):
    u = unit_coords(N)
    b1 = bump_B(N, MID, 0.3)
    b2 = bump_B(N, (0.55, 0.55, 0.55), 0.3)
    phi0 = -10 * b1 * b2 * np.sin(2 * math.pi * u)[None, None, :]
    return phi0, 5 * b1


def _ex7(N):
    phi0 = bump_B(N, (0.4, 0.4, 0.4), 0.2) + bump_B(N, (0.6, 0.6, 0.6), 0.2)
    return phi0, -5 * phi0


EXAMPLES: Dict[str, Example] = {
    "convergence": Example("convergence", 9.0, 2.0, _ex5, [1.0, 2.0],
                           notes="Example 1: n = 200..500 and SP vs DP at t = 1, 2"),
    "blowup": Example("blowup", 1.0, -1.0, _ex2, [1.0, 2.0, 2.5, 2.9, 2.97], stop=1e6,
                      notes="Example 2: |phi| ~ 2 up to t ~ 2, ~ 130 at t = 2.97, then blow-up"),
    "bubble": Example("bubble", 9.0, 2.0, _ex3, [0.21, 0.22, 0.23, 0.4],
                      notes="Example 3: all positive at t = 0.21, sign change at t = 0.22"),
    "long_bubble": Example("long_bubble", 9.0, 2.0, _ex3, [1.0, 2.0, 4.0, 6.0],
                           notes="Example 4: step function with values 0, +-2.12; P(t) -> 0"),
    "no_bubble": Example("no_bubble", 9.0, 2.0, _ex5, [1.0, 2.0, 4.0],
                         notes="Example 5: no zeros inside the support; limit 2.12"),
    "duffing": Example("duffing", 9.0, 2.0, _ex6, [1.0, 4.0],
                       notes="Example 6: non-radial data, positive limit 2.12 at t = 4"),
    "two_bubbles": Example("two_bubbles", 0.1, 0.1, _ex7,
                           [0.07, 0.09, 0.69, 0.8, 1.0, 2.0, 2.15, 3.0], line="diag",
                           notes="Example 7: bubbles at ~0.08, touch at 0.69, inner bubbles at "
                                 "0.8, toroidal at 2.15, gone at 3; values 0, +-1 late"),
    "two_bubbles_t50": Example("two_bubbles_t50", 0.1, 0.1, _ex7,
                               [3.0, 10.0, 20.0, 30.0, 40.0, 50.0], line="diag",
                               notes="Example 7 to t = 50, the paper's longest run (27 h on its "
                                     "GPU); steady state with values 0, +-1"),
}


def line_profile(phi: np.ndarray, which: str) -> np.ndarray:
    N = phi.shape[0]
    if which == "mid":
        return phi[N // 2, N // 2, :].copy()
    i = np.arange(N)
    return phi[i, i, i].copy()


def run_example(ex: Example, n: int = 500, dt: float = 1e-3, prec: int = _lib.FP32,
                eps: float = 1e-6, out_dir: str | None = None) -> dict:
    """Run one example; returns per-time records (max, min, bubbles, integral, P(t))."""
    import torch
    N = n - 1
    phi0, phi1 = ex.init(N)
    mu = math.sqrt(ex.mu2)
    rec = []
    with Solver(N, L_PAPER, mu, ex.lam, _lib.DIRICHLET, prec) as s:
        s.set_initial(torch.from_numpy(phi0).cuda(), torch.from_numpy(phi1).cuda())
        if ex.stop > 0:
            s.set_stop(ex.stop)
        done = 0
        stopped_at = None
        step_secs = 0.0
        for t in ex.times:
            target = int(round(t / dt))
            torch.cuda.synchronize()
            t_start = time.perf_counter()
            st = s.step(target - done, dt) if target > done else _lib.OK
            step_secs += time.perf_counter() - t_start
            done, t_now = s.progress()
            phi = s.read(psi=False)[0]
            d = s.diag(eps=eps)
            a = s.analysis(eps=eps)
            r = {"t": t_now, "max": float(phi.max()), "min": float(phi.min()),
                 "max_abs": d["max_abs_phi"], "bubbles": d["bubble_count"],
                 "n_pos": d["n_pos"], "n_neg": d["n_neg"], "integral_phi": a["integral_phi"],
                 "integral_phi3": a["integral_phi3"], "P": a["laplacian_monitor"],
                 "status": int(st)}
            rec.append(r)
            if out_dir:
                os.makedirs(out_dir, exist_ok=True)
                np.savetxt(os.path.join(out_dir, f"{ex.name}_t{t_now:.4f}_{ex.line}.csv"),
                           line_profile(phi, ex.line), delimiter=",")
            if st != _lib.OK:
                stopped_at = t_now
                break
    return {"example": ex.name, "notes": ex.notes, "n": n, "dt": dt, "records": rec,
            "stopped_at": stopped_at, "stepping_seconds": step_secs,
            "precision": _lib.PREC_NAMES[prec]}


def _mid_line_on_coarse_nodes(phi: np.ndarray, n: int, step: int = 100) -> np.ndarray:
    """phi on the x mid-line at the unit-box nodes u = m / step (m = 1..step-1),
    which every n that is a multiple of `step` has in common."""
    k = n // step
    line = line_profile(phi, "mid")  # unknown i sits at node i + 1
    return line[np.arange(1, step) * k - 1]


def convergence_study(ns: Sequence[int] = (200, 300, 400, 500), times: Sequence[float] = (1.0, 2.0),
                      dt: float = 1e-3) -> dict:
    """Example 1: the mid-line solution for n in `ns` (FP64) against the finest n
    at the common nodes u = m/100, and FP32 against FP64 at the finest n, at
    each time in `times`; also the FP64 / FP32 run-time ratio of the finest
    grid (the paper reports DP about 1.8x the SP run time)."""
    import time
    import torch
    ex = EXAMPLES["convergence"]
    lines: Dict[Tuple[int, int], List[np.ndarray]] = {}
    secs: Dict[Tuple[int, int], float] = {}
    for n in ns:
        for prec in ((_lib.FP64, _lib.FP32) if n == max(ns) else (_lib.FP64,)):
            N = n - 1
            phi0, phi1 = ex.init(N)
            out, done, el = [], 0, 0.0
            with Solver(N, L_PAPER, math.sqrt(ex.mu2), ex.lam, _lib.DIRICHLET, prec) as s:
                s.set_initial(torch.from_numpy(phi0).cuda(), torch.from_numpy(phi1).cuda())
                for t in times:
                    target = int(round(t / dt))
                    torch.cuda.synchronize()
                    t0 = time.perf_counter()
                    s.step(target - done, dt)
                    el += time.perf_counter() - t0
                    done = target
                    out.append(_mid_line_on_coarse_nodes(s.read(psi=False)[0], n))
            lines[(n, prec)] = out
            secs[(n, prec)] = el
    nf = max(ns)
    res = {"times": list(times), "grid_diff": {}, "fp32_vs_fp64": [],
           "fp64_over_fp32_time": secs[(nf, _lib.FP64)] / secs[(nf, _lib.FP32)]}
    for n in ns:
        if n != nf:
            res["grid_diff"][n] = [float(np.max(np.abs(a - b)))
                                   for a, b in zip(lines[(n, _lib.FP64)], lines[(nf, _lib.FP64)])]
    res["fp32_vs_fp64"] = [float(np.max(np.abs(a - b)))
                           for a, b in zip(lines[(nf, _lib.FP32)], lines[(nf, _lib.FP64)])]
    return res


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--out", default=None, help="directory for line profiles and summary.json")
    ap.add_argument("--n", type=int, default=500)
    ap.add_argument("--dt", type=float, default=1e-3)
    ap.add_argument("--only", nargs="*", default=None)
    ap.add_argument("--skip", nargs="*", default=["two_bubbles_t50"],
                    help="examples left out unless named in --only (default: the t = 50 run)")
    ap.add_argument("--convergence", action="store_true",
                    help="also run the Example 1 grid / precision study")
    args = ap.parse_args()
    res = []
    if args.convergence:
        c = convergence_study(dt=args.dt)
        print(json.dumps({"convergence_study": c}), flush=True)
        res.append({"convergence_study": c})
    for name, ex in EXAMPLES.items():
        if args.only and name not in args.only:
            continue
        if not args.only and name in (args.skip or []):
            continue
        r = run_example(ex, args.n, args.dt, out_dir=args.out)
        res.append(r)
        print(json.dumps(r), flush=True)
    if args.out:
        with open(os.path.join(args.out, "summary.json"), "w") as f:
            json.dump(res, f, indent=1)


if __name__ == "__main__":
    main()
