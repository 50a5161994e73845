"""Benchmark of the CMCG Helmholtz solver on the 3D sphere-scattering workload.

Workload (one "step" = one complete CMCG solve, Steps (1)-(6) of the CMCG Algorithm):
  3D unit cube, 7-point stencil, 256^3 intervals (257^3 = 16,974,593 nodes), wave speed
  c(x) = 1 + 0.3 sin(2 pi x) sin(2 pi y) sin(2 pi z), omega = 2 pi * 17.92 (10 points per
  wavelength at c_min = 0.7), sound-soft sphere r = 0.1 at the centre, plane wave
  d = (1/2, 0, sqrt(3)/2) entering through first-order absorbing faces, dt = 0.4 h
  (N = 36 steps per period).  The solve starts from the run-up of Sec. 4.3 (ceil(diam/(T c_min))
  = 45 periods with ramped sources) and stops at a relative CG residual of 5e-10 with respect to
  the zero initial guess, the tolerance at which the solution is within 1e-6 of the plain FP64
  GPU solve.  Precision: FP32 leapfrog fields with FP64 CG vectors, inner products and energy
  functional, inside an FP64 defect-correction loop; the Riesz map is one multigrid V-cycle per
  iteration in flexible CG.

Metric: grid-point leapfrog updates per second (forward and adjoint periods), with solves/s,
the relative error against the plain FP64 GPU solve (tol 1e-10) and per-solve latency.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun each rank runs independent replicas of the solve on its own GPU (the method
has no cross-GPU exchange here); value = all ranks' updates / max-over-ranks time.
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

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "grid-point updates/s and solves/s at rel err 1e-6 vs plain FP64 GPU; p50/p99 latency"
UNIT = "grid-point updates/s"
FALLBACK_HBM_GBS = 6800.0
STEP_BYTES_FP32 = 16  # one step: read y^n, y^{n-1}, kappa; write y^{n+1} (4 B each)
STEP_BYTES_FP64 = 32
PAIR_BYTES_FP32 = 20  # two-step kernel: read y^{n-1}, y^n, kappa; write y^{n+1}, y^{n+2}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=256, help="intervals per axis (default: the full 256^3 workload)")
    ap.add_argument("--tol", type=float, default=5e-10)
    ap.add_argument("--riesz", default="vcycle", choices=["vcycle", "exact"])
    ap.add_argument("--max-iter", type=int, default=0, help="CG iteration cap (profiling runs)")
    ap.add_argument("--runup", type=int, default=-4,
                    help="run-up periods (Sec. 4.3); -k = k domain crossings at c_min, ceil(k diam/(T c_min))")
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp32", "fp64"])
    ap.add_argument("--no-error-check", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    return ap.parse_args()


def workload_config(w, args):
    return {
        "workload": f"3d_sphere_scattering_{w.n[0]}^3",
        "nodes": int(w.num_nodes),
        "stencil": "7-point",
        "wave_speed": "1+0.3 sin(2pi x) sin(2pi y) sin(2pi z)",
        "omega": w.omega,
        "obstacle": "sound-soft sphere r=0.1",
        "incidence": "plane wave d=(1/2,0,sqrt(3)/2) via absorbing BC",
        "dt": "0.4h -> T/N",
        "tol": args.tol,
        "precision": {"mixed": "fp32 stepping + fp64 CG + fp64 defect correction",
                      "fp32": "fp32 stepping + fp64 CG", "fp64": "fp64"}[args.precision],
        "riesz": {"vcycle": "one FP32 multigrid V-cycle per CG iteration (flexible CG)",
                  "exact": "FP64 MG-PCG to 1e-12"}[args.riesz],
        "runup_periods": args.runup,
        "runup": (f"{-args.runup} domain crossings at c_min, ramped sources (Sec. 4.3)" if args.runup < 0
                  else f"{args.runup} periods" if args.runup > 0 else "none"),
        "l2": "inputs larger than L2 (136 MB per FP64 field > 129 MB)",
    }


def tile_config(solver):
    t = list(solver.opts.tile)
    scheme = {2: "two steps per launch", 3: "one step per launch, two z-planes per thread",
              4: "one step per launch, operands staged by TMA bulk copies into a shared-memory ring"}
    return {"tile": t, "step_scheme": scheme.get(t[3], "one step per launch")}


def aggregate_over_ranks(elapsed, updates, device=None):
    """Whole-job figures across ranks: the slowest rank's time and the sum of all updates
    (replicas only: the ranks share nothing but this reduction)."""
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return elapsed, updates
    t = torch.tensor([float(elapsed)], dtype=torch.float64, device=device)
    u = torch.tensor([float(updates)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), float(u.item())


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
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
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


def hbm_peak():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        try:
            d = json.load(open(p))
            for k in ("hbm_gbs", "hbm_GBps", "hbm"):
                if k in d and isinstance(d[k], (int, float)):
                    return float(d[k]), "measured"
        except (OSError, ValueError):
            pass
    return FALLBACK_HBM_GBS, "fallback"


def kernel_traffic(profile, kernel_src_hash):
    """DRAM bytes per launch of a kernel from its committed ncu summary, or None if the kernel
    source changed since the counters were taken."""
    p = os.path.join(ROOT, "profiles", profile)
    if not os.path.exists(p):
        return None
    try:
        d = json.load(open(p))
    except ValueError:
        return None
    if d.get("step_kernel_sha256") != kernel_src_hash:
        return None
    return d.get("dram_bytes_per_launch_full_size")


def kernel_src_hash(name="k_step3d7("):
    """Hash of a kernel's source text in wave.cu (the kernel that ncu counters describe)."""
    fname = "step_bulk.cu" if "bulk" in name else "wave.cu"
    src = open(os.path.join(ROOT, "paper_1903_12522_gb300", "csrc", fname)).read()
    start = src.index(name)
    end = src.index("\n}\n", start) + 2  # the kernel's closing brace
    return hashlib.sha256(src[start:end].encode()).hexdigest()


# ---------------------------------------------------------------------------------------
def cpu_baseline(w, budget_s=15.0):
    """The oracle's leapfrog period on the same grid, timed on the host cores for a bounded
    number of steps; returns updates/s and a description of the sample."""
    from oracle import wave as owave
    from oracle.grid import Discretization

    t0 = time.perf_counter()
    dz = Discretization(w.n, w.h, w.c, w.omega, w.faces, w.dt_target, order=w.order, mask=w.mask)
    setup = time.perf_counter() - t0
    F = dz.load(w.f, w.g)
    y = np.zeros(dz.shape)
    v = np.zeros(dz.shape)
    steps = 0
    t0 = time.perf_counter()
    while True:
        y, v, _ = owave.step(dz, y, v, steps, F)
        steps += 1
        el = time.perf_counter() - t0
        if el >= budget_s or steps >= dz.N:
            break
    ups = steps * dz.size / el
    return {"value": ups, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"{steps} of {dz.N} leapfrog steps of one period on the full {w.shape[0]}^3 grid "
                      f"(numpy/scipy, single thread; setup {setup:.1f}s not timed)"}, steps, el


def run_reference(args):
    ws, rank, local = dist_env()
    if rank != 0:
        return
    from paper_1903_12522_gb300 import workloads as wl

    w = wl.sphere_3d(n=args.n)
    vals = []
    desc = None
    for i in range(args.warmup + args.steps):
        cb, steps, el = cpu_baseline(w, budget_s=5.0)
        if i >= args.warmup:
            vals.append(cb["value"])
            desc = cb
    value = statistics.median(vals)
    ms = 1e3 * (w.num_nodes * 36) / value
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(w, args),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": desc["cores"], "kind": "oracle",
                             "sample": desc["sample"] + "; each step is this bounded sample, ms_per_step scaled to one period"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------------------
def run_ours(args):
    import torch

    from paper_1903_12522_gb300 import cmcg
    from paper_1903_12522_gb300 import workloads as wl

    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    cmcg.load()
    prec = {"mixed": cmcg.MIXED, "fp32": cmcg.FP32, "fp64": cmcg.FP64}[args.precision]
    w = wl.sphere_3d(n=args.n)
    g_host = torch.from_numpy(np.ascontiguousarray(w.g)).pin_memory()
    c_host = torch.from_numpy(np.ascontiguousarray(w.c.ravel())).pin_memory()
    m_host = torch.from_numpy(np.ascontiguousarray(w.mask.ravel())).pin_memory()
    g_dev = g_host.to(dev).reshape(-1)
    rflag = cmcg.FLAG_INEXACT_RIESZ if args.riesz == "vcycle" else 0
    s = cmcg.Solver(w.n, w.h, w.c, w.omega, w.faces, mask=w.mask, precision=prec, dt=w.dt_target,
                    flags=cmcg.FLAG_TIMING | rflag, max_iter=args.max_iter, device=dev, runup_periods=args.runup)
    u = torch.empty(w.num_nodes, dtype=torch.complex128, device=dev)
    stream = s.stream

    def one_solve():
        st = cmcg.Stats()
        code = cmcg.cmcg_solve(s.handle, None, g_dev, args.tol, u, st)
        if code != cmcg.OK and not (args.max_iter and code == cmcg.NOT_CONVERGED):
            raise RuntimeError(f"solve returned {cmcg.cmcg_status_string(code)}")
        return st

    for _ in range(args.warmup):
        one_solve()
    torch.cuda.synchronize()

    # reference: plain FP64 GPU solve to tol 1e-10 (not timed)
    err = None
    u_ref = None
    ref_info = None
    if not args.no_error_check:
        sref = cmcg.Solver(w.n, w.h, w.c, w.omega, w.faces, mask=w.mask, precision=cmcg.FP64, dt=w.dt_target,
                           device=dev)
        t0 = time.perf_counter()
        u_ref, st_ref = sref.solve(None, g_dev, tol=1e-10)
        torch.cuda.synchronize()
        ref_info = {"precision": "fp64 (stepping, CG, exact MG-PCG Riesz to 1e-12)", "tol": 1e-10,
                    "seconds": time.perf_counter() - t0, "cg_iterations": st_ref["iterations"],
                    "updates_per_s": st_ref["point_updates"] / max(time.perf_counter() - t0, 1e-9)}
        sref.close()
        del sref
        torch.cuda.empty_cache()

    clocks = ClockSampler(local)
    if ws > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    stats = []
    lat = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        stats.append(one_solve())
        lat.append(time.perf_counter() - t0)
    ev1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    elapsed = ev0.elapsed_time(ev1) / 1e3
    updates = sum(st.point_updates for st in stats)
    if ws > 1:
        elapsed, updates = aggregate_over_ranks(elapsed, updates, device=dev)
    if u_ref is not None:
        a = u.reshape(w.shape)
        num = torch.linalg.vector_norm(a - u_ref).item()
        den = torch.linalg.vector_norm(u_ref).item()
        err = num / den

    # dominant kernel: the FP32 (or FP64) leapfrog step
    s32 = sum(st.step_seconds_fp32 for st in stats)
    n32 = sum(st.step_launches_fp32 for st in stats)
    s64 = sum(st.step_seconds_fp64 for st in stats)
    n64 = sum(st.step_launches_fp64 for st in stats)
    pairs = s.opts.tile[3] == 2
    tile_cfg = tile_config(s)
    if n32 > 0 and pairs:
        # FP32 3D 7-point periods run their homogeneous steps in pairs (k_step3d7_x2)
        per_launch, bpl, upl = s32 / n32, PAIR_BYTES_FP32, 2
        name, prof, src = "k_step3d7_x2: two FP32 leapfrog steps, 3D 7-point", "step3d7x2_fp32_sphere.json", "k_step3d7_x2("
    elif n32 > 0 and s.opts.tile[3] == 4:
        per_launch, bpl, upl = s32 / n32, STEP_BYTES_FP32, 1
        name, prof, src = ("k_step3d7_bulk<float>: FP32 leapfrog step, 3D 7-point, operands staged by bulk copies",
                           "step3d7bulk_fp32_sphere.json", "k_step3d7_bulk(")
    elif n32 > 0 and s.opts.tile[3] == 3:
        per_launch, bpl, upl = s32 / n32, STEP_BYTES_FP32, 1
        name, prof, src = ("k_step3d7_z2<float>: FP32 leapfrog step, 3D 7-point, two z-planes per thread",
                           "step3d7z2_fp32_sphere.json", "k_step3d7_z2(")
    elif n32 > 0:
        per_launch, bpl, upl = s32 / n32, STEP_BYTES_FP32, 1
        name, prof, src = "k_step3d7<float>: FP32 leapfrog step, 3D 7-point", "step3d7_fp32_sphere.json", "k_step3d7("
    else:
        per_launch, bpl, upl = s64 / max(n64, 1), STEP_BYTES_FP64, 1
        name, prof, src = "k_step3d7<double>: FP64 leapfrog step, 3D 7-point", None, "k_step3d7("
    peak, peak_src = hbm_peak()
    achieved = bpl * w.num_nodes / per_launch / 1e9
    traffic = kernel_traffic(prof, kernel_src_hash(src)) if prof else None
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": traffic, "kernel": name, "algorithmic_bytes_per_node_per_launch": bpl,
                "updates_per_node_per_launch": upl,
                "effective_gbs_at_16B_per_update": STEP_BYTES_FP32 * upl * w.num_nodes / per_launch / 1e9,
                "avg_launch_us": per_launch * 1e6, "peak_source": f"{peak_src} (copy bandwidth)",
                "step_time_share": (s32 + s64) / elapsed if elapsed > 0 else None}

    # e2e through the C ABI with host buffers: copy c, mask, g in; create; solve; copy u out
    e2e = None
    if not args.no_e2e and ws == 1:
        s.close()
        del s
        torch.cuda.empty_cache()
        opts = cmcg.make_options(prec, dt=w.dt_target, flags=cmcg.FLAG_HOST_IO | rflag, runup_periods=args.runup)
        grid = cmcg.make_grid(w.n, w.h)
        ws_t = torch.empty(cmcg.cmcg_workspace_size(grid, opts), dtype=torch.uint8, device=dev)
        c_dev = torch.empty_like(c_host, device=dev)
        m_dev = torch.empty_like(m_host, device=dev)
        u_host = np.empty(w.num_nodes, dtype=np.complex128)
        u_pin = torch.empty(w.num_nodes, dtype=torch.complex128).pin_memory()
        g_np = g_host.numpy().reshape(-1)
        bc = cmcg.BC()
        for f in range(6):
            bc.face[f] = int(w.faces[f])
        st_stream = torch.cuda.current_stream(dev)

        def e2e_step():
            c_dev.copy_(c_host, non_blocking=True)
            m_dev.copy_(m_host, non_blocking=True)
            bc.dirichlet_mask = m_dev.data_ptr()
            h = cmcg.cmcg_create(grid, c_dev, w.omega, bc, opts, ws_t, st_stream.cuda_stream)
            st = cmcg.Stats()
            cmcg.cmcg_solve_host(h, None, g_np, args.tol, u_pin.numpy(), st)
            cmcg.cmcg_destroy(h)
            return st

        e2e_step()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        e2e_updates = 0
        for _ in range(args.steps):
            e2e_updates += e2e_step().point_updates
        torch.cuda.synchronize()
        e_el = time.perf_counter() - t0
        h2d = c_host.numel() * 8 + m_host.numel() + g_host.numel() * 16
        e2e = {"value": e2e_updates / e_el, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
               "d2h_bytes_per_step": int(w.num_nodes * 16),
               "note": "per step: H2D of c, mask, g from pinned memory; cmcg_create; cmcg_solve_host "
                       "(D2H of U inside); cmcg_destroy"}

    if rank != 0:
        if ws > 1:
            dist.destroy_process_group()
        return
    cb = None
    if not args.no_cpu_baseline and ws == 1:
        cb, _, _ = cpu_baseline(w)
    ms_per_step = 1e3 * elapsed / args.steps
    line = {
        "metric": METRIC, "value": updates / elapsed, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": {"mixed": "f32+f64", "fp32": "f32+f64", "fp64": "f64"}[args.precision],
        "data": "synthetic", "config": {**workload_config(w, args), **tile_cfg},
        "solves_per_s": ws * args.steps / elapsed,
        "rel_err_vs_fp64_gpu": err,
        "plain_fp64_gpu_reference": ref_info,
        "latency_ms": {"p50": 1e3 * float(np.percentile(lat, 50)), "p99": 1e3 * float(np.percentile(lat, 99))},
        "cg_iterations": [st.iterations for st in stats],
        "runup_periods_done": [st.runup_periods for st in stats],
        "outer_iterations": [st.outer_iterations for st in stats],
        "riesz_iterations": [st.riesz_iterations for st in stats],
        "periods_per_solve": [st.periods for st in stats],
        "roofline": roofline,
        "cpu_baseline": cb,
        "e2e": e2e,
        "gpu_launches": int(sum(st.kernel_launches for st in stats)),
        "clocks": clk,
    }
    print(json.dumps(line), flush=True)
    if ws > 1:
        dist.destroy_process_group()


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
