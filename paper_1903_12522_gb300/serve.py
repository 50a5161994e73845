"""Batched and served Helmholtz solves on the multi-solve engine (cmcg_engine_*).

  python -m paper_1903_12522_gb300.serve batch [--count 64] [--max-n 1024]
  python -m paper_1903_12522_gb300.serve serve [--requests 40] [--rate 50] [--budget-gb 120]
  python -m paper_1903_12522_gb300.serve batch-compare [--tol 5e-10] [--fp64-tol 5e-10]

batch: the uneven 2D batch -- instances seeded 1000+i, n ~ U{96..1024}, 8-20 points per
  wavelength, smooth random c(x) in [1, 2], one Gaussian source each -- admitted together and
  stepped by one persistent kernel per period; reports solves/s and grid-point updates/s.
batch-compare: the same batch at equal accuracy against FP64 solves of each instance one after
  another (plain, and with the V-cycle Riesz map and the run-up), errors against FP64 to 1e-10.
serve: Poisson arrivals (seeded) of a 70 % 2D (n ~ U{128..512}) / 30 % 3D (n ~ U{64..256})
  request mix, 10-16 points per wavelength, smooth random c, one random source, tol 1e-6.
  A request is admitted when its workspace (cmcg_workspace_size) fits the memory budget and a
  slot is free; solves that arrive while others run join the next tick (continuous batching)
  and leave when they finish.  Reports p50/p99 latency (arrival to result) and solves/s.

Inputs are synthetic and seeded; the 3D smooth random fields are generated on the GPU (torch
FFT) because host generation is slower than the arrival rate.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
if os.path.dirname(HERE) not in sys.path:
    sys.path.insert(0, os.path.dirname(HERE))

from paper_1903_12522_gb300 import autotune  # noqa: E402
from paper_1903_12522_gb300 import cmcg  # noqa: E402
from paper_1903_12522_gb300 import workloads as wl  # noqa: E402


# ---- request recipe ----------------------------------------------------------------------
def smooth_field_torch(shape, seed, device, corr_len=0.1, lo=1.0, hi=2.0):
    """Smooth Gaussian random field on the device: white noise, Gaussian filter, affine map."""
    import torch

    gen = torch.Generator(device=device)
    gen.manual_seed(int(seed))
    noise = torch.randn(shape, generator=gen, device=device, dtype=torch.float64)
    n = max(shape) - 1
    sig = corr_len * n
    spec = torch.fft.fftn(noise)
    filt = torch.ones(shape, device=device, dtype=torch.float64)
    for ax, m in enumerate(shape):
        fr = torch.fft.fftfreq(m, device=device, dtype=torch.float64)
        gk = torch.exp(-2.0 * (math.pi * sig * fr) ** 2)
        sh = [1] * len(shape)
        sh[ax] = m
        filt = filt * gk.reshape(sh)
    field = torch.fft.ifftn(spec * filt).real
    fmin, fmax = field.min(), field.max()
    return lo + (hi - lo) * (field - fmin) / (fmax - fmin)


def gaussian_source_torch(n, h, center, sigma, device):
    import torch

    d = len(n)
    r2 = 0.0
    for a in range(d):
        x = torch.arange(n[a] + 1, device=device, dtype=torch.float64) * h
        sh = [1] * d
        sh[d - 1 - a] = n[a] + 1
        r2 = r2 + ((x - center[a]) ** 2).reshape(sh)
    return torch.exp(-r2 / (2.0 * sigma * sigma)).to(torch.complex128)


class Request:
    def __init__(self, rid, arrival, dim, n, ppw, src, seed):
        self.rid, self.arrival, self.dim, self.n, self.ppw, self.src, self.seed = rid, arrival, dim, n, ppw, src, seed
        self.h = 1.0 / n
        self.omega = 2.0 * math.pi * 1.0 / (ppw * self.h)  # c_min = 1
        self.dt_target = 0.9 * self.h / (math.sqrt(dim) * 2.0)  # c_max = 2
        self.admitted = None
        self.finished = None
        self.stats = None
        self.rejected = False

    def grid(self):
        return (self.n,) * self.dim

    def build(self, device):
        shape = (self.n + 1,) * self.dim
        c = smooth_field_torch(shape, self.seed, device)
        f = gaussian_source_torch(self.grid(), self.h, self.src, 0.4 * self.ppw * self.h, device)
        return c, f


def poisson_requests(count, rate, seed=5, two_d=(128, 512), three_d=(64, 256), frac_2d=0.7, ppw=(10.0, 16.0)):
    rng = np.random.Generator(np.random.PCG64(seed))
    t = 0.0
    out = []
    for i in range(count):
        t += rng.exponential(1.0 / rate)
        dim = 2 if rng.random() < frac_2d else 3
        lo, hi = two_d if dim == 2 else three_d
        n = int(rng.integers(lo, hi + 1))
        p = float(rng.uniform(*ppw))
        src = tuple(rng.uniform(0.2, 0.8, size=dim))
        out.append(Request(i, t, dim, n, p, src, seed * 100000 + i))
    return out


# ---- engine driver -------------------------------------------------------------------------
def make_solver(req, c, precision, stream, runup=0):
    faces = (cmcg.BC_ABC,) * 6
    return cmcg.Solver(req.grid(), req.h, c, req.omega, faces, precision=precision, dt=req.dt_target,
                       flags=cmcg.FLAG_INEXACT_RIESZ, stream=stream, runup_periods=runup)


def workspace_bytes(req, precision):
    return cmcg.cmcg_workspace_size(cmcg.make_grid(req.grid(), req.h),
                                    cmcg.make_options(precision, flags=cmcg.FLAG_INEXACT_RIESZ))


class WallClock:
    """Arrivals, admissions and completions on the wall clock (seconds since start)."""

    def __init__(self):
        self.t0 = time.perf_counter()

    def now(self):
        return time.perf_counter() - self.t0

    def idle_until(self, t):
        time.sleep(max(0.0, min(t - self.now(), 0.05)))

    def ticked(self):
        pass


class TickClock:
    """A simulated clock that advances by a fixed time per engine tick and jumps to the next
    arrival when nothing runs.  Admission then depends only on the request stream and the
    tick count, not on how fast the GPU or the host happens to be, so a run is repeatable."""

    def __init__(self, tick_s):
        self.tick_s = float(tick_s)
        self.t = 0.0

    def now(self):
        return self.t

    def idle_until(self, t):
        self.t = max(self.t, t)

    def ticked(self):
        self.t += self.tick_s


def serve(requests, budget_bytes, max_slots=64, precision=cmcg.MIXED, tol=1e-6, device="cuda", log=None,
          keep_results=False, stream=None, runup=0, tick_s=None):
    """Run the request stream; returns per-request records and totals.  Arrivals follow the
    wall clock, or with tick_s a simulated clock that advances tick_s seconds per engine tick
    (latencies are then in simulated time; wall_s and the rates stay on the wall clock)."""
    import torch

    eng = cmcg.Engine(max_slots=max_slots, stream=stream, shape=autotune.lookup_engine("mix"))
    stream = eng.stream
    clock = TickClock(tick_s) if tick_s else WallClock()
    queue = list(requests)
    waiting = []
    running = {}
    used = 0
    done = []
    rejected = []
    t0 = time.perf_counter()
    updates = 0
    while queue or waiting or running:
        now = clock.now()
        while queue and queue[0].arrival <= now:
            waiting.append(queue.pop(0))
        # admission: first fit in arrival order by workspace bytes and free slots; a request
        # whose workspace alone exceeds the budget could never start and is rejected
        for req in list(waiting):
            if len(running) >= max_slots:
                break
            nb = workspace_bytes(req, precision)
            if nb > budget_bytes:
                waiting.remove(req)
                req.rejected = True
                rejected.append(req)
                continue
            if used + nb > budget_bytes:
                continue
            c, f = req.build(device)
            s = make_solver(req, c, precision, stream, runup)
            slot = eng.submit(s, f, None, tol)
            req.admitted = clock.now()
            running[slot] = (req, s, nb)
            used += nb
            waiting.remove(req)
        if not running:
            if queue:
                clock.idle_until(queue[0].arrival)
            continue
        finished = eng.tick()
        clock.ticked()
        for slot in finished:
            req, s, nb = running.pop(slot)
            u, st = eng.result(slot)
            req.finished = clock.now()
            req.stats = st
            if keep_results:
                req.result = u.clone()
            updates += st["point_updates"]
            used -= nb
            s.close()
            done.append(req)
            if log:
                log(req)
    wall = time.perf_counter() - t0
    info = eng.info()
    eng.close()
    lat = np.array([r.finished - r.arrival for r in done])
    latency = None if len(done) == 0 else {
        "p50": 1e3 * float(np.percentile(lat, 50)), "p99": 1e3 * float(np.percentile(lat, 99)),
        "mean": 1e3 * float(lat.mean())}
    return {
        "requests": len(done),
        "rejected": len(rejected),
        "wall_s": wall,
        "solves_per_s": len(done) / wall,
        "updates_per_s": updates / wall,
        "latency_ms": latency,
        "queue_ms_mean": None if len(done) == 0 else 1e3 * float(np.mean([r.admitted - r.arrival for r in done])),
        "status_ok": int(sum(1 for r in done if r.stats["status"] == cmcg.OK)),
        "ticks": info["ticks"],
        "graph_builds": info["graph_builds"],
    }


def batch(count=64, max_n=None, precision=cmcg.MIXED, tol=1e-6, device="cuda", runup=0):
    """The uneven 2D batch solved together; returns totals."""
    import torch

    eng = cmcg.Engine(max_slots=count, shape=autotune.lookup_engine("batch2d"))
    stream = eng.stream
    ws = batch_instances(count, max_n)
    solvers = [cmcg.Solver(w.n, w.h, w.c, w.omega, w.faces, precision=precision, dt=w.dt_target,
                           flags=cmcg.FLAG_INEXACT_RIESZ, stream=stream, runup_periods=runup) for w in ws]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for s, w in zip(solvers, ws):
        eng.submit(s, w.f, None, tol)
    res = eng.run_all()
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    info = eng.info()
    eng.close()
    sts = [st for _, st in res.values()]
    return {
        "instances": count,
        "nodes_total": int(sum(w.num_nodes for w in ws)),
        "wall_s": wall,
        "solves_per_s": count / wall,
        "updates_per_s": sum(st["point_updates"] for st in sts) / wall,
        "iterations": {"min": min(st["iterations"] for st in sts), "max": max(st["iterations"] for st in sts)},
        "status_ok": sum(1 for st in sts if st["status"] == cmcg.OK),
        "ticks": info["ticks"],
        "graph_builds": info["graph_builds"],
    }


def batch_instances(count, max_n=None):
    ws = []
    for i in range(count):
        w = wl.random_2d_instance(i)
        if max_n is not None and w.n[0] > max_n:
            w = wl.random_2d_instance(i, n=max_n)
        ws.append(w)
    return ws


def batch_compare(count=64, max_n=None, tol=5e-10, fp64_tol=5e-10, fp64_tuned_tol=1e-10, runup=-2, device="cuda"):
    """The uneven 2D batch at equal accuracy: the mixed-precision engine batch against the same
    instances solved one after another by the plain FP64 GPU CMCG (FP64 stepping, exact Riesz
    map, no run-up) and by the FP64 solver with the V-cycle Riesz map and the run-up; every
    field's error against a plain FP64 solve to tol 1e-10 (not timed)."""
    import torch

    ws = batch_instances(count, max_n)

    def rel(u, r):
        return float(torch.linalg.vector_norm(u.reshape(-1) - r.reshape(-1)) / torch.linalg.vector_norm(r))

    def fp64_solve(w, tol_, flags=0, ru=0):
        s = cmcg.Solver(w.n, w.h, w.c, w.omega, w.faces, precision=cmcg.FP64, dt=w.dt_target, flags=flags,
                        runup_periods=ru)
        u, st = s.solve(w.f, None, tol=tol_)
        s.close()
        return u, st

    refs = [fp64_solve(w, 1e-10)[0] for w in ws]
    out = {"instances": count, "nodes_total": int(sum(w.num_nodes for w in ws)), "tol_reference": 1e-10}
    for key, tol_, flags, ru in (("fp64_plain", fp64_tol, 0, 0),
                                 ("fp64_tuned", fp64_tuned_tol, cmcg.FLAG_INEXACT_RIESZ, runup)):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        errs = []
        for w, r in zip(ws, refs):
            u, st = fp64_solve(w, tol_, flags, ru)
            errs.append(rel(u, r))
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        out[key] = {"tol": tol_, "wall_s": wall, "solves_per_s": count / wall, "max_rel_err": max(errs),
                    "median_rel_err": float(np.median(errs))}
    eng = cmcg.Engine(max_slots=count, shape=autotune.lookup_engine("batch2d"))
    stream = eng.stream
    solvers = [cmcg.Solver(w.n, w.h, w.c, w.omega, w.faces, precision=cmcg.MIXED, dt=w.dt_target,
                           flags=cmcg.FLAG_INEXACT_RIESZ, stream=stream, runup_periods=runup) for w in ws]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    slots = [eng.submit(s, w.f, None, tol) for s, w in zip(solvers, ws)]
    res = eng.run_all()
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    eng.close()
    errs = [rel(res[sl][0], r) for sl, r in zip(slots, refs)]
    out["mixed_batch"] = {"tol": tol, "wall_s": wall, "solves_per_s": count / wall, "max_rel_err": max(errs),
                          "median_rel_err": float(np.median(errs)),
                          "status_ok": sum(1 for sl in slots if res[sl][1]["status"] == cmcg.OK)}
    for key in ("fp64_plain", "fp64_tuned"):
        out[f"speedup_vs_{key}"] = out["mixed_batch"]["solves_per_s"] / out[key]["solves_per_s"]
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("mode", choices=["batch", "serve", "batch-compare"])
    ap.add_argument("--count", type=int, default=64)
    ap.add_argument("--max-n", type=int, default=None)
    ap.add_argument("--requests", type=int, default=40)
    ap.add_argument("--rate", type=float, default=50.0)
    ap.add_argument("--budget-gb", type=float, default=120.0)
    ap.add_argument("--tol", type=float, default=1e-6)
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp32"])
    ap.add_argument("--runup", type=int, default=-2,
                    help="run-up periods per solve (Sec. 4.2.3; -k = k domain crossings; mixed precision only)")
    ap.add_argument("--max-3d", type=int, default=256)
    ap.add_argument("--fp64-tol", type=float, default=5e-10, help="batch-compare: tolerance of the plain FP64 solves")
    ap.add_argument("--fp64-tuned-tol", type=float, default=1e-10,
                    help="batch-compare: tolerance of the FP64 solves with the V-cycle Riesz map and the run-up")
    ap.add_argument("--tick-s", type=float, default=None,
                    help="serve: arrivals on a simulated clock advancing this much per tick (repeatable runs)")
    a = ap.parse_args()
    prec = cmcg.MIXED if a.precision == "mixed" else cmcg.FP32
    if a.mode == "batch":
        out = batch(a.count, a.max_n, prec, a.tol, runup=a.runup)
    elif a.mode == "batch-compare":
        out = batch_compare(a.count, a.max_n, a.tol, a.fp64_tol, a.fp64_tuned_tol, runup=a.runup)
    else:
        reqs = poisson_requests(a.requests, a.rate, three_d=(64, a.max_3d))
        out = serve(reqs, int(a.budget_gb * 1e9), precision=prec, tol=a.tol, runup=a.runup, tick_s=a.tick_s)
    print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()
