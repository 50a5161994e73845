"""Benchmark of the CMCG Helmholtz solver on the 3D sphere-scattering workload.

Workload (one "step" = one complete CMCG solve, Steps (1)-(6) of the CMCG Algorithm):
  3D unit cube, 7-point stencil, 256^3 intervals (257^3 = 16,974,593 nodes), wave speed
  c(x) = 1 + 0.3 sin(2 pi x) sin(2 pi y) sin(2 pi z), omega = 2 pi * 17.92 (10 points per
  wavelength at c_min = 0.7), sound-soft sphere r = 0.1 at the centre, plane wave
  d = (1/2, 0, sqrt(3)/2) entering through first-order absorbing faces, dt = 0.4 h
  (N = 36 steps per period).  The solve starts from the run-up of Sec. 4.2.3 (ceil(diam/(T c_min))
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
                    help="run-up periods (Sec. 4.2.3); -k = k domain crossings at c_min, ceil(k diam/(T c_min))")
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp32", "fp64"])
    ap.add_argument("--no-error-check", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64-comparators", action="store_true")
    ap.add_argument("--no-l2-kappa", action="store_true", help="do not keep kappa resident in L2 (CMCG_FLAG_L2_KAPPA)")
    # profiling entry points (instead of the benchmark line): pieces of the solver timed with
    # CUDA events on a workload, for ncu captures and the measurements quoted in the design notes
    ap.add_argument("--profile", default=None,
                    choices=["period", "adjoint", "solve", "riesz", "fo-period", "fo-adjoint", "fo-solve", "stream",
                             "obstacles"],
                    help="period/adjoint/riesz/solve/fo-*: time that call --reps times; stream: copy and "
                         "3-read/1-write bandwidth of PyTorch's own kernels; obstacles: CMCG against the "
                         "do-nothing solver on the square obstacle and the cavity (Sec. 4.2)")
    ap.add_argument("--workload", default="sphere", choices=["sphere", "layered", "gauss2d"])
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--tile", type=int, nargs=4, default=None, help="cmcg_options.tile (default: autotuned)")
    ap.add_argument("--inner-tol", type=float, default=0.0)
    ap.add_argument("--filter", action="store_true", help="recover U by the fundamental-frequency filter")
    ap.add_argument("--l2-kappa", action="store_true", help="--profile: keep kappa resident in L2 (CMCG_FLAG_L2_KAPPA)")
    ap.add_argument("--fp64-plain-tol", type=float, default=5e-10,
                    help="tolerance of the plain FP64 comparator (chosen so that its error is about 1e-6)")
    ap.add_argument("--fp64-tuned-tol", type=float, default=1e-10,
                    help="tolerance of the tuned FP64 comparator (chosen so that its error is about 1e-6)")
    return ap.parse_args()


def workload_config(w):
    """The workload itself (the same in both arms); how each arm computes is in "method"."""
    return {
        "workload": f"3d_sphere_scattering_{w.n[0]}^3",
        "nodes": int(w.num_nodes),
        "stencil": "7-point",
        "wave_speed": "1+0.3 sin(2pi x) sin(2pi y) sin(2pi z)",
        "omega": w.omega,
        "obstacle": "sound-soft sphere r=0.1",
        "incidence": "plane wave d=(1/2,0,sqrt(3)/2) via absorbing BC",
        "dt": "0.4h -> T/N",
        "l2": "inputs larger than L2 (136 MB per FP64 field > 129 MB)",
    }


def method_config(args):
    return {
        "step": "one complete CMCG solve (Steps (1)-(6) of the CMCG Algorithm)",
        "tol": args.tol,
        "precision": {"mixed": "fp32 stepping + fp64 CG + fp64 defect correction",
                      "fp32": "fp32 stepping + fp64 CG", "fp64": "fp64"}[args.precision],
        "riesz": {"vcycle": "one FP32 multigrid V-cycle per CG iteration (flexible CG)",
                  "exact": "FP64 MG-PCG to 1e-12"}[args.riesz],
        "runup_periods": args.runup,
        "runup": (f"{-args.runup} domain crossings at c_min, ramped sources (Sec. 4.2.3)" if args.runup < 0
                  else f"{args.runup} periods" if args.runup > 0 else "none"),
        "l2_kappa": "off" if getattr(args, "no_l2_kappa", False) else
                    "FP32 kappa kept in an L2 set-aside across steps (CMCG_FLAG_L2_KAPPA)",
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
    """Hash of a kernel's source text (the kernel that ncu counters describe)."""
    fname = "step_bulk.cu" if "bulk" in name else ("step_pair.cu" if "pair" in name else "wave.cu")
    src = open(os.path.join(ROOT, "paper_1903_12522_gb300", "csrc", fname)).read()
    start = src.index(name)
    end = src.index("\n}\n", start) + 2  # the kernel's closing brace
    return hashlib.sha256(src[start:end].encode()).hexdigest()


# ---------------------------------------------------------------------------------------
# The oracle on the host cores: the plain FP64 CPU implementation (numpy/scipy, written from
# the paper), timed as it stands.  It is single-threaded, so "all cores" means independent
# replicas of the same bounded sample, one process per core (spawned: no CUDA state is
# inherited), as many as the host memory holds.
ORACLE_BYTES_PER_NODE = 600  # resident set of one oracle replica per grid node (9.6 GB at 257^3)


def host_cpu():
    """(logical cores, CPU model) of this host."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.split(":")[0].strip() in ("Model name", "Model"):
                model = line.split(":", 1)[1].strip()
                if not model.isdigit():
                    break
    except (OSError, subprocess.SubprocessError):
        pass
    if not model:
        try:
            for line in open("/proc/cpuinfo"):
                if line.lower().startswith(("model name", "cpu part")):
                    model = line.split(":", 1)[1].strip()
                    break
        except OSError:
            pass
    return os.cpu_count() or 1, model or "unknown"


def host_mem_available():
    avail = None
    try:
        for line in open("/proc/meminfo"):
            if line.startswith("MemAvailable:"):
                avail = int(line.split()[1]) * 1024
    except (OSError, ValueError):
        pass
    try:
        lim = open("/sys/fs/cgroup/memory.max").read().strip()
        if lim.isdigit():
            avail = min(avail or int(lim), int(lim))
    except OSError:
        pass
    return avail


def oracle_replica_count(num_nodes):
    cores, _ = host_cpu()
    mem = host_mem_available()
    per = ORACLE_BYTES_PER_NODE * num_nodes
    by_mem = cores if mem is None else int(0.6 * mem // per)
    return max(1, min(cores, by_mem))


def _oracle_replica(conn, n):
    """Spawned child: build the workload and the oracle's discretisation, then answer each
    request of the parent with (steps, seconds) of leapfrog steps run for that many seconds."""
    from oracle import wave as owave
    from oracle.grid import Discretization
    from paper_1903_12522_gb300 import workloads as wl

    w = wl.sphere_3d(n=n)
    dz = Discretization(w.n, w.h, w.c, w.omega, w.faces, w.dt_target, order=w.order, mask=w.mask)
    F = dz.load(w.f, w.g)
    y = np.zeros(dz.shape)
    v = np.zeros(dz.shape)
    k = 0
    conn.send((dz.size, dz.N))
    while True:
        budget = conn.recv()
        if budget is None:
            break
        steps = 0
        t0 = time.perf_counter()
        while True:
            y, v, _ = owave.step(dz, y, v, k, F)
            k += 1
            steps += 1
            el = time.perf_counter() - t0
            if el >= budget:
                break
        conn.send((steps, el))
    conn.close()


class OracleReplicas:
    """P spawned oracle replicas of the full workload; each round runs every replica for a
    bounded time at once and returns (updates, seconds) with seconds = the slowest replica."""

    def __init__(self, n, procs):
        import multiprocessing as mp

        for var in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
            os.environ[var] = "1"  # one thread per replica
        ctx = mp.get_context("spawn")
        self.conns, self.procs = [], []
        for _ in range(procs):
            a, b = ctx.Pipe()
            p = ctx.Process(target=_oracle_replica, args=(b, n), daemon=True)
            p.start()
            self.conns.append(a)
            self.procs.append(p)
        t0 = time.perf_counter()
        ready = [c.recv() for c in self.conns]
        self.setup_s = time.perf_counter() - t0
        self.size, self.N = ready[0]

    def round(self, budget_s):
        for c in self.conns:
            c.send(float(budget_s))
        res = [c.recv() for c in self.conns]
        return sum(st for st, _ in res) * self.size, max(el for _, el in res), [st for st, _ in res]

    def close(self):
        for c in self.conns:
            try:
                c.send(None)
            except (OSError, BrokenPipeError):
                pass
        for p in self.procs:
            p.join(timeout=30)


def oracle_description(procs, budget_s, size, N, setup_s):
    cores, model = host_cpu()
    return (f"{procs} independent replica(s) of the oracle (plain FP64 numpy/scipy leapfrog, single-threaded "
            f"each, one per core) on the full {size:,}-node grid; each timed round runs every replica's "
            f"leapfrog steps for {budget_s:.0f} s (a bounded sample of the {N}-step period); host: {cores} "
            f"logical cores, {model}; setup {setup_s:.0f} s not timed")


def cpu_baseline(w, budget_s=5.0, rounds=2):
    """The oracle's leapfrog steps on the same grid, on all host cores (replicas)."""
    procs = oracle_replica_count(w.num_nodes)
    rep = OracleReplicas(w.n[0], procs)
    try:
        rep.round(1.0)  # warm-up
        upd, el = 0.0, 0.0
        for _ in range(rounds):
            u, e, _ = rep.round(budget_s)
            upd += u
            el += e
    finally:
        rep.close()
    cores, model = host_cpu()
    return {"value": upd / el, "unit": UNIT, "cores": procs, "kind": "oracle", "cpu": model, "nproc": cores,
            "per_core_value": upd / el / procs,
            "sample": oracle_description(procs, budget_s, rep.size, rep.N, rep.setup_s) + f"; {rounds} rounds"}


def run_reference(args):
    """The reference arm: the oracle, as it stands, on the host cores (no GPU).  Each step is
    one bounded round of every replica; ms_per_step is the time of that round."""
    ws, rank, local = dist_env()
    if rank != 0:
        return
    from paper_1903_12522_gb300 import workloads as wl

    w = wl.sphere_3d(n=args.n)
    procs = oracle_replica_count(w.num_nodes)
    budget = 4.0
    rep = OracleReplicas(args.n, procs)
    try:
        for _ in range(args.warmup):
            rep.round(budget)
        upd, el, steps = 0.0, 0.0, []
        for _ in range(args.steps):
            u, e, st = rep.round(budget)
            upd += u
            el += e
            steps.append(st)
    finally:
        rep.close()
    value = upd / el
    cores, model = host_cpu()
    desc = oracle_description(procs, budget, rep.size, rep.N, rep.setup_s)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(w),
            "method": {"step": "one bounded round of oracle leapfrog steps (FP64, CPU) on every replica",
                       "leapfrog_steps_per_replica_per_step": steps},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": procs, "kind": "oracle", "cpu": model,
                             "nproc": cores, "per_core_value": value / procs, "sample": desc},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def target_comparison(comparators, solves_per_s, err):
    """Solves/s of this solve against the FP64 GPU solves at (about) the same accuracy."""
    if not comparators:
        return None
    out = {"target_rel_err": 1e-6, "this_solve": {"solves_per_s": solves_per_s, "rel_err_vs_fp64_gpu": err}}
    for key, c in comparators.items():
        out[key] = c
        out[f"speedup_vs_{key}"] = solves_per_s / c["solves_per_s"]
    return out


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
    l2flag = 0 if args.no_l2_kappa else cmcg.FLAG_L2_KAPPA
    s = cmcg.Solver(w.n, w.h, w.c, w.omega, w.faces, mask=w.mask, precision=prec, dt=w.dt_target,
                    flags=cmcg.FLAG_TIMING | rflag | l2flag, max_iter=args.max_iter, device=dev,
                    runup_periods=args.runup)
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

    # The plain FP64 GPU CMCG (FP64 stepping and CG, exact MG-PCG Riesz map, zero initial
    # guess): to tol 1e-10 it is the accuracy reference; at a looser tolerance, and in its best
    # FP64 form (one V-cycle Riesz map, the run-up), it is the comparator of the solves/s target
    # at relative error 1e-6.  Each is one solve, timed on its own (outside the timed region).
    def fp64_solve(tol, flags, runup):
        sref = cmcg.Solver(w.n, w.h, w.c, w.omega, w.faces, mask=w.mask, precision=cmcg.FP64, dt=w.dt_target,
                           flags=flags, runup_periods=runup, device=dev)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        u_c, st_c = sref.solve(None, g_dev, tol=tol)
        torch.cuda.synchronize()
        el = time.perf_counter() - t0
        sref.close()
        del sref
        torch.cuda.empty_cache()
        return u_c, st_c, el

    def rel_err(a, b):
        return (torch.linalg.vector_norm(a.reshape(-1) - b.reshape(-1)) / torch.linalg.vector_norm(b)).item()

    err = None
    u_ref = None
    ref_info = None
    comparators = {}
    if not args.no_error_check:
        u_ref, st_ref, el = fp64_solve(1e-10, 0, 0)
        ref_info = {"precision": "fp64 (stepping, CG, exact MG-PCG Riesz to 1e-12), no run-up", "tol": 1e-10,
                    "seconds": el, "cg_iterations": st_ref["iterations"],
                    "updates_per_s": st_ref["point_updates"] / el}
        if not args.no_fp64_comparators:
            for key, tol, fl, ru, desc in (
                    ("fp64_plain", args.fp64_plain_tol, 0, 0,
                     "plain FP64 GPU CMCG: FP64 stepping and CG, exact MG-PCG Riesz map, no run-up"),
                    ("fp64_tuned", args.fp64_tuned_tol, cmcg.FLAG_INEXACT_RIESZ, args.runup,
                     "FP64 GPU CMCG with this solver's other speed-ups: one V-cycle Riesz map (flexible CG) "
                     "and the same run-up")):
                u_c, st_c, el = fp64_solve(tol, fl, ru)
                comparators[key] = {"what": desc, "tol": tol, "seconds_per_solve": el, "solves_per_s": 1.0 / el,
                                    "rel_err_vs_fp64_gpu": rel_err(u_c, u_ref), "cg_iterations": st_c["iterations"],
                                    "runup_periods": st_c["runup_periods"]}
                del u_c
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
        # FP32 3D 7-point periods run their homogeneous steps in pairs (k_step3d7_pair)
        per_launch, bpl, upl = s32 / n32, PAIR_BYTES_FP32, 2
        name, prof, src = ("k_step3d7_pair: two FP32 leapfrog steps, 3D 7-point", "step3d7pair_fp32_sphere.json",
                           "k_step3d7_pair(")
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
        opts = cmcg.make_options(prec, dt=w.dt_target, flags=cmcg.FLAG_HOST_IO | rflag | l2flag,
                                 runup_periods=args.runup)
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
        # a created stream, as a C-ABI caller would pass: CG iterations replay as CUDA graphs and
        # the L2 window applies (neither is available on the legacy default stream)
        st_stream = torch.cuda.Stream(dev)

        def e2e_step():
            with torch.cuda.stream(st_stream):
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
               "note": "per step, on a created stream: H2D of c, mask, g from pinned memory; cmcg_create; "
                       "cmcg_solve_host (D2H of U inside); cmcg_destroy"}

    if rank != 0:
        if ws > 1:
            dist.destroy_process_group()
        return
    cb = None
    if not args.no_cpu_baseline and ws == 1:
        cb = cpu_baseline(w)
    ms_per_step = 1e3 * elapsed / args.steps
    line = {
        "metric": METRIC, "value": updates / elapsed, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": {"mixed": "f32+f64", "fp32": "f32+f64", "fp64": "f64"}[args.precision],
        "data": "synthetic", "config": workload_config(w), "method": {**method_config(args), **tile_cfg},
        "solves_per_s": ws * args.steps / elapsed,
        "rel_err_vs_fp64_gpu": err,
        "plain_fp64_gpu_reference": ref_info,
        "vs_fp64_at_equal_accuracy": target_comparison(comparators, ws * args.steps / elapsed, err),
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


# ---------------------------------------------------------------------------------------
# Profiling entry points (--profile): not part of the benchmark line.
def run_profile(a):
    import torch

    from paper_1903_12522_gb300 import cmcg
    from paper_1903_12522_gb300 import workloads as wl

    if a.profile == "obstacles":
        return profile_obstacles(a.n)
    if a.profile == "stream":
        return profile_stream(a.n, a.reps)
    prec = {"fp32": cmcg.FP32, "fp64": cmcg.FP64, "mixed": cmcg.MIXED}[a.precision]
    w = {"sphere": wl.sphere_3d, "layered": wl.layered_3d, "gauss2d": wl.gaussian_2d}[a.workload](n=a.n)
    fo = a.profile.startswith("fo-")
    flags = cmcg.FLAG_FIRST_ORDER if fo else (cmcg.FLAG_INEXACT_RIESZ if a.riesz == "vcycle" else 0)
    if a.filter:
        flags |= cmcg.FLAG_FILTER
    if a.l2_kappa:
        flags |= cmcg.FLAG_L2_KAPPA
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
        if a.profile == "period":
            s.wave_period(y0, v0, f, g)
        elif a.profile == "adjoint":
            s.adjoint_period(y0, v0)
        elif a.profile == "riesz":
            s.riesz(y0)
        elif a.profile == "fo-period":
            s.fo_period(x)
        elif a.profile == "fo-adjoint":
            s.fo_adjoint_period(x)
        else:
            _, st = s.solve(f, g, tol=a.tol)
            print(f"  solve: iterations={st['iterations']} periods={st['periods']} runup={st['runup_periods']} "
                  f"rel={st['rel_residual']:.2e} status={st['status']}", flush=True)
        e1.record(s.stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        ups = (N * w.num_nodes / (ms * 1e-3)) if a.profile in ("period", "adjoint", "fo-period", "fo-adjoint") \
            else float("nan")
        print(f"{a.profile} n={a.n} {a.precision} rep={r} ms={ms:.3f} updates/s={ups:.4g}", flush=True)


def _axis_weights(n):
    # trapezoidal weights of the node-based L2 norm along one axis (1/2 at both ends)
    a = np.ones(n + 1)
    a[0] = a[-1] = 0.5
    return a


def profile_obstacles(n, ells=(10, 25, 50, 100, 200, 400)):
    """Sec. 4.2 on the GPU: for each l, the error of the do-nothing state after l ramped periods
    (Eq. AP_SOLUTION) and of the CMCG iterate after l iterations from zero, both against a
    converged FP64 CMCG solve, with each one's relative periodicity misfit sqrt(J) / ||g_S||."""
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


def profile_stream(n, reps):
    """Bandwidth calibration with PyTorch's own elementwise kernels on (n+1)^3 FP32 arrays: a
    copy (1 read + 1 write) and p += a * b in place (3 reads + 1 write, the access mix of the
    one-step leapfrog kernel without its neighbour loads).  Prints GB/s per pattern."""
    import torch

    m = (n + 1) ** 3
    a, b, p, q = [torch.rand(m, device="cuda", dtype=torch.float32) for _ in range(4)]
    flush = torch.empty(256 * 1024 * 1024 // 4, device="cuda", dtype=torch.float32)
    out = {}
    for name, fn, nbytes in (("copy_1r1w", lambda: q.copy_(a), 8 * m),
                             ("addcmul_3r1w", lambda: p.addcmul_(a, b), 16 * m)):
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


def main():
    args = parse()
    if args.profile:
        run_profile(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
