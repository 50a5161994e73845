"""Kernel exerciser for profiling: runs the solver's pieces on a synthetic workload.

  python -m paper_1903_12522_gb300.probe period --n 256 --precision fp32 --reps 3
  python -m paper_1903_12522_gb300.probe solve  --n 128 --precision mixed --max-iter 4
  python -m paper_1903_12522_gb300.probe period --workload layered --n 512 --precision fp32

"period" runs cmcg_wave_period (start kernel, N-1 leapfrog steps, end kernel) on random
initial data of the 3D sphere workload; "solve" runs cmcg_solve with an iteration cap.
Prints one timing line per repetition (CUDA events on the solver's stream).

  python -m paper_1903_12522_gb300.probe obstacles --n 128

"obstacles" prints the comparison of Sec. 4.2 on the convex square and the semi-open cavity:
for each l, the error of the do-nothing state after l periods (Eq. AP_SOLUTION, ramped
sources) and of the CMCG iterate after l iterations (zero initial guess), both against a
converged FP64 CMCG solve, plus each one's relative periodicity misfit sqrt(J) / ||g_S||
(Sec. 4.2).
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
    ap.add_argument("mode", choices=["period", "adjoint", "solve", "riesz", "obstacles", "fo-period", "fo-adjoint",
                                     "fo-solve", "stream"])
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
    ap.add_argument("--filter", action="store_true", help="recover U by the fundamental-frequency filter")
    a = ap.parse_args()
    if a.mode == "obstacles":
        return obstacles(a.n)
    if a.mode == "stream":
        return stream(a.n, a.reps)
    prec = {"fp32": cmcg.FP32, "fp64": cmcg.FP64, "mixed": cmcg.MIXED}[a.precision]
    w = {"sphere": wl.sphere_3d, "layered": wl.layered_3d, "gauss2d": wl.gaussian_2d}[a.workload](n=a.n)
    fo = a.mode.startswith("fo-")
    flags = cmcg.FLAG_FIRST_ORDER if fo else (cmcg.FLAG_INEXACT_RIESZ if a.inexact else 0)
    if a.filter:
        flags |= cmcg.FLAG_FILTER
    s = cmcg.Solver(w.n, w.h, w.c, w.omega, w.faces, mask=w.mask, order=w.order, precision=prec, dt=w.dt_target,
                    max_iter=a.max_iter, flags=flags, runup_periods=a.runup, tile=None if fo else a.tile,
                    inner_tol=a.inner_tol)
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
    if fo:
        x = torch.randn((w.dim + 1) * w.num_nodes, generator=gen, device="cuda", dtype=torch.float64)
    for r in range(a.reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(s.stream)
        if a.mode == "period":
            s.wave_period(y0, v0, f, g)
        elif a.mode == "adjoint":
            s.adjoint_period(y0, v0)
        elif a.mode == "riesz":
            s.riesz(y0)
        elif a.mode == "fo-period":
            s.fo_period(x)
        elif a.mode == "fo-adjoint":
            s.fo_adjoint_period(x)
        else:
            _, st = s.solve(f, g, tol=a.tol)
            print(f"  solve: iterations={st['iterations']} periods={st['periods']} runup={st['runup_periods']} "
                  f"rel={st['rel_residual']:.2e} status={st['status']}", flush=True)
        e1.record(s.stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        ups = (N * w.num_nodes / (ms * 1e-3)) if a.mode in ("period", "adjoint", "fo-period", "fo-adjoint") \
            else float("nan")
        print(f"{a.mode} n={a.n} {a.precision} rep={r} ms={ms:.3f} updates/s={ups:.4g}", flush=True)


def obstacles(n: int, ells=(10, 25, 50, 100, 200, 400)):
    import json
    import math

    import torch

    from paper_1903_12522_gb300 import cmcg
    from paper_1903_12522_gb300 import workloads as wl

    for cavity in (False, True):
        w = wl.square_obstacle_2d(n=n, cavity=cavity)
        wts = torch.as_tensor(np.outer(_axis_weights(n), _axis_weights(n)) * w.h ** 2, device="cuda").reshape(-1)

        def solver(**kw):
            return cmcg.Solver(w.n, w.h, w.c, w.omega, w.faces, mask=w.mask, precision=cmcg.FP64, dt=w.dt_target,
                               **kw)

        ref, st = solver().solve(None, w.g, tol=1e-12)
        norm = math.sqrt(float(torch.sum(wts * ref.reshape(-1).abs() ** 2)))
        g2 = np.abs(w.g) ** 2  # ||g_S||_{L2(Gamma_S)}: trapezoidal rule along each absorbing side
        t = _axis_weights(n) * w.h
        fnorm = math.sqrt(float(t @ g2[0] + t @ g2[-1] + t @ g2[:, 0] + t @ g2[:, -1]))

        def err(u):
            return math.sqrt(float(torch.sum(wts * (u.reshape(-1) - ref.reshape(-1)).abs() ** 2))) / norm

        rows = []
        for ell in ells:
            u_dn, s_dn = solver(flags=cmcg.FLAG_NO_CG, runup_periods=ell).solve(None, w.g, tol=1e-6)
            u_cg, s_cg = solver(max_iter=ell).solve(None, w.g, tol=1e-14)
            rows.append({"l": ell, "do_nothing_err": err(u_dn), "cmcg_err": err(u_cg),
                         "do_nothing_misfit": math.sqrt(max(s_dn["J_final"], 0.0)) / fnorm,
                         "cmcg_misfit": math.sqrt(max(s_cg["J_final"], 0.0)) / fnorm})
        print(json.dumps({"workload": w.name, "reference_cg_iterations": st["iterations"], "rows": rows}), flush=True)


def stream(n: int, reps: int):
    """Bandwidth calibration with PyTorch's own elementwise kernels on (n+1)^3 FP32 arrays: a
    copy (1 read + 1 write) and p += a * b in place (3 reads + 1 write, the access mix of the
    one-step leapfrog kernel without its neighbour loads).  Prints GB/s per pattern."""
    import json

    import torch

    m = (n + 1) ** 3
    a, b, p, q = [torch.rand(m, device="cuda", dtype=torch.float32) for _ in range(4)]
    flush = torch.empty(256 * 1024 * 1024 // 4, device="cuda", dtype=torch.float32)
    out = {}
    for name, fn, nbytes in (("copy_1r1w", lambda: q.copy_(a), 8 * m), ("addcmul_3r1w", lambda: p.addcmul_(a, b), 16 * m)):
        for _ in range(3):
            fn()
        times = []
        for _ in range(max(reps, 5)):
            flush.zero_()  # evict L2 between runs
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            fn()
            e1.record()
            torch.cuda.synchronize()
            times.append(e0.elapsed_time(e1) * 1e-3)
        t = sorted(times)[len(times) // 2]
        out[name] = {"us": t * 1e6, "GB_s": nbytes / t / 1e9}
    print(json.dumps({"n": n, "nodes": m, "median": out}), flush=True)


def _axis_weights(n: int) -> np.ndarray:
    # trapezoidal weights of the node-based L2 norm along one axis (1/2 at both ends)
    a = np.ones(n + 1)
    a[0] = a[-1] = 0.5
    return a


if __name__ == "__main__":
    main()
