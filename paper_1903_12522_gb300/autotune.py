"""Autotuner for the leapfrog kernels' launch shapes, cached to JSON per grid class.

  python -m paper_1903_12522_gb300.autotune --dim 3 --n 256 --precision fp32

For a grid class (dimension, size bucket = the power of two nearest the largest interval
count, precision) it times the homogeneous adjoint period (one-step and two-step kernels) for
every candidate launch shape in cmcg_options.tile and records the fastest in
autotune_cache.json next to this file.  Solver() looks the class up when no tile is given.
"""
from __future__ import annotations

import argparse
import json
import math
import os

HERE = os.path.dirname(os.path.abspath(__file__))
CACHE = os.path.join(HERE, "autotune_cache.json")

def candidates_3d():
    """cmcg_options.tile candidates: scheme 1 (one z-plane per loop trip) and 3 (two, or four
    with tile[2] = 4), tile[0] = z-planes per thread; scheme 2 (two steps per launch), tile[1] = z-planes per block and
    tile[2] = tile height (the two shapes that ranked best on 257^3 and 513^3); scheme 4
    (bulk-copy staging), tile[0] = planes per CTA and tile[1] = band rows (0 = automatic)."""
    out = []
    for scheme in (1, 3):
        out += [(zc, 0, 0, scheme) for zc in (8, 16, 32)]
    out += [(zc, 0, 4, 3) for zc in (8, 16, 32)]  # scheme 3 with four planes per loop iteration
    out += [(16, 12, 16, 2), (16, 24, 16, 2)]
    out += [(zc, ty, 0, 4) for zc in (0, 16, 32, 64) for ty in (0, 4, 8)]
    return out


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


def lookup(dim, n, precision):
    """Tuned cmcg_options.tile for the class, or None (library defaults)."""
    entry = _load().get(size_class(dim, n, precision))
    return None if entry is None else tuple(entry["tile"])


def tune(dim, n, precision, reps=5):
    import torch

    from . import cmcg
    from . import workloads as wl

    assert dim == 3, "the launch-shape knobs are those of the 3D kernels"
    w = wl.sphere_3d(n=n)
    act = 1.0 - w.mask.astype("float64")
    a, b = [torch.as_tensor(x * act, device="cuda").reshape(-1) for x in wl.random_fields(w.shape, 2, 17)]
    results = []
    for tile in candidates_3d():
        s = cmcg.Solver(w.n, w.h, w.c, w.omega, w.faces, mask=w.mask, precision=precision, dt=w.dt_target, tile=tile)
        s.adjoint_period(a, b)  # warm-up
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(s.stream)
        for _ in range(reps):
            s.adjoint_period(a, b)
        e1.record(s.stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / reps
        results.append((ms, tile))
        s.close()
    results.sort()
    best_ms, best = results[0]
    cache = _load()
    cache[size_class(dim, n, precision)] = {"tile": list(best), "ms_per_adjoint_period": best_ms,
                                            "candidates": len(results), "worst_ms": results[-1][0]}
    json.dump(cache, open(CACHE, "w"), indent=1, sort_keys=True)
    return best, best_ms, results


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--dim", type=int, default=3)
    ap.add_argument("--n", type=int, nargs="+", default=[256])
    ap.add_argument("--precision", default="fp32", choices=["fp32", "mixed", "fp64"])
    a = ap.parse_args()
    from . import cmcg

    prec = {"fp32": cmcg.FP32, "mixed": cmcg.MIXED, "fp64": cmcg.FP64}[a.precision]
    for n in a.n:
        best, ms, res = tune(a.dim, n, prec)
        print(json.dumps({"class": size_class(a.dim, n, prec), "tile": best, "ms": ms, "worst_ms": res[-1][0],
                          "all": [[round(t, 4), list(c)] for t, c in res]}))


if __name__ == "__main__":
    main()
