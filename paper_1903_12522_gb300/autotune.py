"""Autotuner for the leapfrog kernels' launch shapes, cached to JSON per workload class.

  python -m paper_1903_12522_gb300.autotune --dim 3 --n 256 --precision fp32
  python -m paper_1903_12522_gb300.autotune --dim 2 --n 128 512 1024 --precision fp32
  python -m paper_1903_12522_gb300.autotune --engine batch2d mix

Single solves: for a grid class (dimension, size bucket = the power of two nearest the largest
interval count, precision) it times the homogeneous adjoint period for every candidate step
scheme and launch shape in cmcg_options.tile and records the fastest in autotune_cache.json
next to this file; Solver() looks the class up when no tile is given.  The 3D candidates
include the temporal-blocking depth (one or two leapfrog steps per sweep: schemes 1/3/4/5/6
against scheme 2) and the number of planes in flight of the staged kernel (scheme 6).

Engine: for a batch class ("batch2d": uneven 2D instances; "mix": 2D and 3D requests) it
times engine ticks of a fixed set of solves in their inner iterations for every launch shape
of the batched persistent step kernel (resident blocks per SM, z-planes per work item of 3D
grids) and records the fastest; serve.py passes it to the engine.
"""
from __future__ import annotations

import argparse
import json
import math
import os

HERE = os.path.dirname(os.path.abspath(__file__))
CACHE = os.path.join(HERE, "autotune_cache.json")


def candidates_3d():
    """cmcg_options.tile candidates on 3D 7-point grids: scheme 1 (one z-plane per loop trip)
    and 3 (two, or four with tile[2] = 4), tile[0] = z-planes per thread; scheme 2 (two steps
    per launch: temporal-blocking depth 2), tile[0] = planes staged ahead, tile[1] = z-planes
    per block and tile[2] = tile height; scheme 4 (bulk-copy staging), tile[0] = planes per CTA and tile[1] = band rows (0 =
    automatic); scheme 5 (one float4 of the flat index per thread); scheme 6 (staged by
    asynchronous copies), tile[1] = band rows, tile[2] = planes in flight."""
    out = []
    for scheme in (1, 3):
        out += [(zc, 0, 0, scheme) for zc in (8, 16, 32)]
    out += [(zc, 0, 4, 3) for zc in (8, 16, 32)]  # scheme 3 with four planes per loop iteration
    out += [(2, 16, 0, 2), (3, 16, 0, 2), (2, 32, 0, 2)]  # scheme 2: planes staged ahead, z-planes per block
    out += [(zc, ty, 0, 4) for zc in (0, 16, 32, 64) for ty in (0, 4, 8)]
    out += [(0, 0, 0, 5)]
    out += [(0, ty, depth, 6) for ty in (0, 1, 2, 3, 4) for depth in (2, 3)]
    return out


def candidates_2d():
    """2D 5-point grids: the generic one-step kernel and the vector form."""
    return [(0, 0, 0, 1), (0, 0, 0, 5)]


def engine_candidates():
    """(resident blocks per SM of the batched kernel, 0 = as many as fit; z-planes per work item
    of 3D grids)."""
    return [(b, z) for b in (0, 2, 4) for z in (8, 16, 32)]


def size_class(dim, n, precision):
    # FP32 and mixed solves run the same FP32 step kernels
    kind = "fp64" if int(precision) == 0 else "fp32"
    return f"d{dim}_n{2 ** int(round(math.log2(max(int(n), 2))))}_{kind}"


def _load():
    if os.path.exists(CACHE):
        try:
            return json.load(open(CACHE))
        except ValueError:
            return {}
    return {}


def _store(key, entry):
    cache = _load()
    cache[key] = entry
    json.dump(cache, open(CACHE, "w"), indent=1, sort_keys=True)


def lookup(dim, n, precision):
    """Tuned cmcg_options.tile for the class, or None (library defaults)."""
    entry = _load().get(size_class(dim, n, precision))
    return None if entry is None else tuple(entry["tile"])


def lookup_engine(kind):
    """Tuned (blocks per SM, z-planes) of the batched kernel for a batch class, or None."""
    entry = _load().get(f"engine_{kind}")
    return None if entry is None else tuple(entry["shape"])


def _time_adjoint(s, a, b, reps):
    import torch

    s.adjoint_period(a, b)  # warm-up
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(s.stream)
    for _ in range(reps):
        s.adjoint_period(a, b)
    e1.record(s.stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def tune(dim, n, precision, reps=5, rounds=2):
    import torch

    from . import cmcg
    from . import workloads as wl

    w = wl.sphere_3d(n=n) if dim == 3 else wl.gaussian_2d(n=n)
    act = 1.0 if w.mask is None else 1.0 - w.mask.astype("float64")
    a, b = [torch.as_tensor(x * act, device="cuda").reshape(-1) for x in wl.random_fields(w.shape, 2, 17)]
    cands = candidates_3d() if dim == 3 else candidates_2d()
    best = {}
    for _ in range(rounds):  # the best of several rounds, the candidates interleaved
        for tile in cands:
            s = cmcg.Solver(w.n, w.h, w.c, w.omega, w.faces, mask=w.mask, precision=precision, dt=w.dt_target,
                            tile=tile)
            ms = _time_adjoint(s, a, b, reps)
            best[tile] = min(best.get(tile, float("inf")), ms)
            s.close()
    results = sorted((ms, tile) for tile, ms in best.items())
    best_ms, best_tile = results[0]
    _store(size_class(dim, n, precision), {"tile": list(best_tile), "ms_per_adjoint_period": best_ms,
                                           "candidates": len(results), "worst_ms": results[-1][0]})
    return best_tile, best_ms, results


def engine_mix(kind):
    """The fixed solve set of a batch class: small enough to tune in seconds, shaped like it."""
    from . import workloads as wl

    if kind == "batch2d":
        return [wl.random_2d_instance(i, n=min(wl.random_2d_instance(i).n[0], 512)) for i in range(16)]
    out = [wl.random_2d_instance(i, n=128 + 24 * i) for i in range(8)]
    out += [wl.sphere_3d(n=n, obstacle=False) for n in (48, 64, 96)]
    return out


def tune_engine(kind, ticks=12, warm=4):
    import torch

    from . import cmcg

    ws = engine_mix(kind)
    results = []
    for shape in engine_candidates():
        stream = torch.cuda.Stream()
        eng = cmcg.Engine(max_slots=len(ws), stream=stream, shape=shape)
        solvers = [cmcg.Solver(w.n, w.h, w.c, w.omega, w.faces, mask=w.mask, precision=cmcg.FP32, dt=w.dt_target,
                               flags=cmcg.FLAG_INEXACT_RIESZ, stream=stream, max_iter=100000) for w in ws]
        for s, w in zip(solvers, ws):
            eng.submit(s, w.f, w.g, 1e-15)  # none finishes inside the timed ticks
        for _ in range(warm):
            eng.tick()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(ticks):
            eng.tick()
        e1.record(stream)
        torch.cuda.synchronize()
        results.append((e0.elapsed_time(e1) / ticks, shape))
        eng.close()
        for s in solvers:
            s.close()
    results.sort()
    best_ms, best = results[0]
    _store(f"engine_{kind}", {"shape": list(best), "ms_per_tick": best_ms, "candidates": len(results),
                              "worst_ms": results[-1][0], "solves": len(ws)})
    return best, best_ms, results


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--dim", type=int, default=3)
    ap.add_argument("--n", type=int, nargs="+", default=[256])
    ap.add_argument("--precision", default="fp32", choices=["fp32", "mixed", "fp64"])
    ap.add_argument("--engine", nargs="*", default=None, choices=["batch2d", "mix"],
                    help="tune the batched kernel of these batch classes instead")
    a = ap.parse_args()
    from . import cmcg

    if a.engine:
        for kind in a.engine:
            best, ms, res = tune_engine(kind)
            print(json.dumps({"class": f"engine_{kind}", "shape": best, "ms_per_tick": ms, "worst_ms": res[-1][0],
                              "all": [[round(t, 4), list(c)] for t, c in res]}), flush=True)
        return
    prec = {"fp32": cmcg.FP32, "mixed": cmcg.MIXED, "fp64": cmcg.FP64}[a.precision]
    for n in a.n:
        best, ms, res = tune(a.dim, n, prec)
        print(json.dumps({"class": size_class(a.dim, n, prec), "tile": best, "ms": ms, "worst_ms": res[-1][0],
                          "all": [[round(t, 4), list(c)] for t, c in res]}), flush=True)


if __name__ == "__main__":
    main()
