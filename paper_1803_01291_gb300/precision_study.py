"""The precision study on the benchmark workloads: each reduced-precision path
against the FP64 GPU path (which the tests hold to the FP64 oracle at 1e-11).

* GRF 512^3 periodic, lambda in {0.5, 1, 2}, to t = 6 (308 steps): relative
  max-norm error of phi and psi for FP32 (compensated state), BF16-stored
  stage values and plain FP32; sign masks (bits that differ from FP64's) and
  bubble counts; throughput of each path.
* Gaussians 256^3 zero-Dirichlet to t = 5, diagnostics every 0.5 time units:
  FP32 error and bubble counts against FP64 at every diagnostic time.
* Focusing blow-up 1024^3 (lambda = -1), stop at max|phi| > 1e6: the step and
  time at which FP32 and FP64 stop, and their throughput.

Run:  python -m paper_1803_01291_gb300.precision_study [--out FILE] [--skip-blowup]
"""
from __future__ import annotations

import argparse
import json
import time
from typing import Dict

import numpy as np

from . import _lib
from .solver import Solver

NAMES = {_lib.FP64: "fp64", _lib.FP32: "fp32", _lib.BF16: "bf16", _lib.FP32_PLAIN: "fp32_plain"}


def _solver(prob, prec):
    import torch
    s = Solver(prob.N, prob.L, prob.mu, prob.lam, prob.bc, prec)
    s.set_initial(torch.from_numpy(prob.phi0).cuda(), torch.from_numpy(prob.phi1).cuda())
    return s


def _timed_steps(s, n, dt):
    import torch
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    st = s.step(n, dt)
    return st, time.perf_counter() - t0


def _mask_diff(a: dict, b: dict) -> int:
    """Number of grid points whose strict sign differs between two diagnostics."""
    x = np.bitwise_xor(a["pos_mask"], b["pos_mask"]) | np.bitwise_xor(a["neg_mask"], b["neg_mask"])
    return int(np.unpackbits(x.view(np.uint8)).sum())


def grf_study(lams=(0.5, 1.0, 2.0), N: int = 512, eps: float = 1e-6) -> list:
    import hbe_inputs as hi
    rows = []
    for lam in lams:
        prob = hi.grf_problem(N, lam=lam, seed=0)
        res: Dict[int, dict] = {}
        for prec in (_lib.FP64, _lib.FP32, _lib.BF16, _lib.FP32_PLAIN):
            with _solver(prob, prec) as s:
                st, secs = _timed_steps(s, prob.nsteps, prob.dt)
                phi, psi, t = s.read()
                d = s.diag(eps=eps, masks=True)
            res[prec] = {"phi": phi, "psi": psi, "diag": d, "secs": secs, "status": int(st), "t": t}
        ref = res[_lib.FP64]
        sp, sq = np.max(np.abs(ref["phi"])), np.max(np.abs(ref["psi"]))
        row = {"lambda": lam, "t": ref["t"], "steps": prob.nsteps,
               "fp64": {"gpoint_steps_per_s": N ** 3 * prob.nsteps / ref["secs"] / 1e9,
                        "bubble_count": ref["diag"]["bubble_count"]}}
        for prec in (_lib.FP32, _lib.BF16, _lib.FP32_PLAIN):
            r = res[prec]
            row[NAMES[prec]] = {
                "phi_rel_maxnorm": float(np.max(np.abs(r["phi"] - ref["phi"])) / sp),
                "psi_rel_maxnorm": float(np.max(np.abs(r["psi"] - ref["psi"])) / sq),
                "sign_points_differing": _mask_diff(r["diag"], ref["diag"]),
                "bubble_count": r["diag"]["bubble_count"],
                "gpoint_steps_per_s": N ** 3 * prob.nsteps / r["secs"] / 1e9}
        rows.append(row)
        print(json.dumps({"grf": row}), flush=True)
    return rows


def gaussians_study(N: int = 256, eps: float = 1e-6) -> list:
    import hbe_inputs as hi
    prob = hi.gaussians_problem(N)
    marks = [int(round(0.5 * j / prob.dt)) for j in range(1, 11)]
    marks[-1] = prob.nsteps
    runs = {}
    for prec in (_lib.FP64, _lib.FP32):
        with _solver(prob, prec) as s:
            done, out = 0, []
            for m in marks:
                s.step(m - done, prob.dt)
                done = m
                out.append((s.read(psi=False)[0], s.diag(eps=eps, masks=True), s.progress()[1]))
            runs[prec] = out
    rows = []
    for (a, da, t), (b, db, _) in zip(runs[_lib.FP32], runs[_lib.FP64]):
        rows.append({"t": t, "fp32_phi_rel_maxnorm": float(np.max(np.abs(a - b)) / np.max(np.abs(b))),
                     "bubbles_fp64": db["bubble_count"], "bubbles_fp32": da["bubble_count"],
                     "sign_points_differing": _mask_diff(da, db)})
    print(json.dumps({"gaussians": rows}), flush=True)
    return rows


def blowup_study(N: int = 1024) -> dict:
    import torch
    import hbe_inputs as hi
    prob = hi.blowup_problem(N)
    out = {}
    for prec in (_lib.FP32, _lib.FP64):
        with _solver(prob, prec) as s:
            s.set_stop(1e6)
            st, secs = _timed_steps(s, prob.nsteps, prob.dt)
            n, t = s.progress()
            out[NAMES[prec]] = {"status": _lib.STATUS_NAMES.get(int(st), int(st)), "steps": n,
                                "blowup_time": t, "max_abs_phi": s.diag()["max_abs_phi"],
                                "gpoint_steps_per_s": N ** 3 * n / secs / 1e9}
        torch.cuda.empty_cache()
    out["dt"] = prob.dt
    print(json.dumps({"blowup": out}), flush=True)
    return out


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--out", default=None)
    ap.add_argument("--skip-blowup", action="store_true")
    args = ap.parse_args()
    rep = {"grf_512": grf_study(), "gaussians_256": gaussians_study()}
    if not args.skip_blowup:
        rep["blowup_1024"] = blowup_study()
    if args.out:
        with open(args.out, "w") as f:
            json.dump(rep, f, indent=1)


if __name__ == "__main__":
    main()
