"""Kernel exerciser for profiling: runs the solver's pieces on a synthetic workload.

  python -m paper_1903_12522_gb300.probe period --n 256 --precision fp32 --reps 3
  python -m paper_1903_12522_gb300.probe solve  --n 128 --precision mixed --max-iter 4
  python -m paper_1903_12522_gb300.probe period --workload layered --n 512 --precision fp32

"period" runs cmcg_wave_period (start kernel, N-1 leapfrog steps, end kernel) on random
initial data of the 3D sphere workload; "solve" runs cmcg_solve with an iteration cap.
Prints one timing line per repetition (CUDA events on the solver's stream).
"""
from __future__ import annotations

import argparse
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(HERE))


def main():
    import torch

    from paper_1903_12522_gb300 import cmcg
    from paper_1903_12522_gb300 import workloads as wl

    ap = argparse.ArgumentParser()
    ap.add_argument("mode", choices=["period", "adjoint", "solve", "riesz"])
    ap.add_argument("--n", type=int, default=256)
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp64", "mixed"])
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--max-iter", type=int, default=4)
    ap.add_argument("--tol", type=float, default=1e-6)
    ap.add_argument("--workload", default="sphere", choices=["sphere", "layered", "gauss2d"])
    ap.add_argument("--inexact", action="store_true", help="one V-cycle per CG iteration as the Riesz map")
    ap.add_argument("--runup", type=int, default=0)
    ap.add_argument("--tile", type=int, nargs=4, default=None, help="cmcg_options.tile (default: autotuned)")
    ap.add_argument("--inner-tol", type=float, default=0.0)
    a = ap.parse_args()
    prec = {"fp32": cmcg.FP32, "fp64": cmcg.FP64, "mixed": cmcg.MIXED}[a.precision]
    w = {"sphere": wl.sphere_3d, "layered": wl.layered_3d, "gauss2d": wl.gaussian_2d}[a.workload](n=a.n)
    s = cmcg.Solver(w.n, w.h, w.c, w.omega, w.faces, mask=w.mask, order=w.order, precision=prec, dt=w.dt_target,
                    max_iter=a.max_iter, flags=cmcg.FLAG_INEXACT_RIESZ if a.inexact else 0, runup_periods=a.runup,
                    tile=a.tile, inner_tol=a.inner_tol)
    act = 1.0 if w.mask is None else 1.0 - w.mask.astype(np.float64)
    gen = torch.Generator(device="cuda")
    gen.manual_seed(7)
    y0, v0 = [torch.randn(w.num_nodes, generator=gen, device="cuda", dtype=torch.float64) for _ in range(2)]
    if w.mask is not None:
        m = torch.as_tensor(act, device="cuda").reshape(-1)
        y0, v0 = y0 * m, v0 * m
    g = None if w.g is None else torch.as_tensor(w.g, device="cuda").reshape(-1)
    f = None if w.f is None else torch.as_tensor(w.f, device="cuda").reshape(-1)
    N = s.info["steps_per_period"]
    for r in range(a.reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(s.stream)
        if a.mode == "period":
            s.wave_period(y0, v0, f, g)
        elif a.mode == "adjoint":
            s.adjoint_period(y0, v0)
        elif a.mode == "riesz":
            s.riesz(y0)
        else:
            _, st = s.solve(f, g, tol=a.tol)
            print(f"  solve: iterations={st['iterations']} periods={st['periods']} runup={st['runup_periods']} "
                  f"rel={st['rel_residual']:.2e} status={st['status']}", flush=True)
        e1.record(s.stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        ups = (N * w.num_nodes / (ms * 1e-3)) if a.mode in ("period", "adjoint") else float("nan")
        print(f"{a.mode} n={a.n} {a.precision} rep={r} ms={ms:.3f} updates/s={ups:.4g}", flush=True)


if __name__ == "__main__":
    main()
