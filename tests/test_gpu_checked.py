"""The compiled-in bounds checks (libcmcg_checked.so, built with -DCMCG_CHECKED), standing in
for a sanitizer: every kernel family that derives node indices from its launch coordinates
runs on small grids with ragged tails, every boundary type, both stencil orders and every
step scheme, and must record no out-of-range index while its results still match the oracle.
The checked library runs in a child process (one library per process); the parent checks
that the normal library reports the checks as not compiled in.  Also: two runs of the same
solve are bitwise equal (every reduction has a fixed order)."""
import os
import subprocess
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_1903_12522_gb300 import cmcg  # noqa: E402
from paper_1903_12522_gb300 import workloads as wl  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r'''
import math
import numpy as np
import torch
from oracle import direct, wave
from oracle.grid import Discretization
from paper_1903_12522_gb300 import cmcg
from paper_1903_12522_gb300 import workloads as wl

ABC, NEU, DIR = wl.ABC, wl.NEUMANN, wl.DIRICHLET
lib = cmcg.load()
assert lib._name == cmcg.LIB_CHECKED_PATH, lib._name
done = []


def clean(tag):
    code, count, site, index = cmcg.cmcg_check_status()
    assert code == cmcg.OK, (tag, code)
    assert count == 0, f"{tag}: {count} failed bounds checks, first at site {site}, index {index}"
    done.append(tag)


def rel(a, b):
    return float(np.linalg.norm((np.asarray(a) - b).ravel()) / max(np.linalg.norm(np.ravel(b)), 1e-300))


def dz_of(w):
    return Discretization(w.n, w.h, w.c, w.omega, w.faces, w.dt_target, order=w.order, mask=w.mask)


def odd_3d():
    n = (13, 11, 15)
    h = 1.0 / 15
    rng = np.random.Generator(np.random.PCG64(12))
    c = 1.0 + 0.5 * rng.random((16, 12, 14))
    f = wl.gaussian_source(n, h, (0.4, 0.3, 0.5), 0.1).astype(np.complex128)
    return wl.Workload(name="odd3d", n=n, h=h, c=c, omega=7.0, faces=(ABC, ABC, NEU, ABC, ABC, ABC),
                       dt_target=0.3 * h / 1.5, f=f)


def odd_2d():
    n = (37, 29)
    h = 1.0 / 37
    rng = np.random.Generator(np.random.PCG64(13))
    c = 1.0 + rng.random((30, 38))
    g = (rng.standard_normal((30, 38)) + 1j * rng.standard_normal((30, 38))).astype(np.complex128)
    return wl.Workload(name="odd2d", n=n, h=h, c=c, omega=11.0, faces=(ABC,) * 4 + (NEU, NEU),
                       dt_target=0.4 * h / 2.0, mask=wl.sphere_mask(n, h, (0.5, 0.4), 0.12), g=g)


clean("load")
cases = [wl.gaussian_2d(n=40), odd_2d(), odd_3d(), wl.sphere_3d(n=24), wl.layered_3d(n=16)]
schemes_3d = [None, (0, 0, 0, 1), (3, 0, 0, 3), (5, 0, 4, 3), (0, 0, 0, 2), (1, 3, 8, 2), (0, 0, 0, 4),
              (0, 0, 0, 5), (0, 0, 0, 6)]
for w in cases:
    dz = dz_of(w)
    rng = np.random.Generator(np.random.PCG64(5))
    y0 = rng.standard_normal(dz.shape) * dz.act
    v0 = rng.standard_normal(dz.shape) * dz.act
    yF, vF = wave.period(dz, y0, v0, dz.load(w.f, w.g))
    q0, q1 = wave.transposed_period(dz, y0, v0)
    tiles = schemes_3d if (w.dim == 3 and w.order == 2) else [None, (0, 0, 0, 1), (0, 0, 0, 5)]
    for precision, tol in ((cmcg.FP64, 1e-12), (cmcg.FP32, 2e-5)):
        for tile in (tiles if precision == cmcg.FP32 else [None]):
            s = cmcg.Solver(w.n, w.h, w.c, w.omega, w.faces, mask=w.mask, order=w.order, precision=precision,
                            dt=w.dt_target, tile=tile)
            uT, uV = s.wave_period(y0, v0, w.f, w.g)
            assert rel(uT.cpu().numpy(), yF) <= tol and rel(uV.cpu().numpy(), vF) <= tol, (w.name, tile)
            g0, g1 = s.adjoint_period(y0, v0)
            assert rel(g0.cpu().numpy(), q0) <= tol and rel(g1.cpu().numpy(), q1) <= tol, (w.name, tile)
            s.close()
            clean(f"{w.name} periods {precision} {tile}")
    # solves: the exact and the V-cycle Riesz maps (multigrid kernels), mixed precision, run-up
    U = direct.solve(dz, dz.load(w.f, w.g))
    for precision, flags, runup, tol, bound in ((cmcg.FP64, 0, 0, 1e-13, 1e-10),
                                                (cmcg.MIXED, cmcg.FLAG_INEXACT_RIESZ, -2, 1e-9, 1e-6)):
        s = cmcg.Solver(w.n, w.h, w.c, w.omega, w.faces, mask=w.mask, order=w.order, precision=precision,
                        dt=w.dt_target, flags=flags, runup_periods=runup)
        u, st = s.solve(w.f, w.g, tol=tol)
        err = math.sqrt(float(np.sum(dz.W * np.abs(u.cpu().numpy() - U) ** 2) / np.sum(dz.W * np.abs(U) ** 2)))
        assert err <= bound, (w.name, precision, err, st)
        s.close()
        clean(f"{w.name} solve {precision}")
# the batched persistent step kernel
stream = torch.cuda.Stream()
ws = [wl.gaussian_2d(n=40), odd_2d(), wl.sphere_3d(n=16)]
eng = cmcg.Engine(max_slots=len(ws), stream=stream)
solvers = [cmcg.Solver(w.n, w.h, w.c, w.omega, w.faces, mask=w.mask, order=w.order, precision=cmcg.MIXED,
                       dt=w.dt_target, flags=cmcg.FLAG_INEXACT_RIESZ, stream=stream) for w in ws]
slots = [eng.submit(s, w.f, w.g, 1e-9) for s, w in zip(solvers, ws)]
res = eng.run_all()
for w, sl in zip(ws, slots):
    u, st = res[sl]
    dz = dz_of(w)
    U = direct.solve(dz, dz.load(w.f, w.g))
    err = math.sqrt(float(np.sum(dz.W * np.abs(u.cpu().numpy() - U) ** 2) / np.sum(dz.W * np.abs(U) ** 2)))
    assert st["status"] == cmcg.OK and err <= 1e-6, (w.name, err, st)
eng.close()
for s in solvers:
    s.close()
clean("engine batch")
print("CHECKED OK", len(done))
'''


def test_checked_build_finds_no_out_of_range_index():
    from paper_1903_12522_gb300 import build

    if not os.path.exists(cmcg.LIB_CHECKED_PATH):
        build.build(checked=True)
    env = dict(os.environ, CMCG_CHECKED="1", PYTHONPATH=ROOT + os.pathsep + os.environ.get("PYTHONPATH", ""))
    r = subprocess.run([sys.executable, "-c", CHILD], cwd=ROOT, env=env, capture_output=True, text=True,
                       timeout=1500)
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-3000:]
    assert "CHECKED OK" in r.stdout, r.stdout[-2000:]


def test_normal_build_has_no_checks():
    code, count, site, index = cmcg.cmcg_check_status()
    assert code == cmcg.ERR_UNSUPPORTED and count == 0 and site == -1


def test_two_runs_are_bitwise_equal():
    # fixed-order reductions: the same mixed-precision solve (V-cycle Riesz map, run-up) twice
    # gives the same bits (the determinism check that stands in for a race detector)
    w = wl.sphere_3d(n=24)
    outs = []
    for _ in range(2):
        s = cmcg.Solver(w.n, w.h, w.c, w.omega, w.faces, mask=w.mask, order=w.order, precision=cmcg.MIXED,
                        dt=w.dt_target, flags=cmcg.FLAG_INEXACT_RIESZ, runup_periods=-2)
        u, st = s.solve(w.f, w.g, tol=1e-10)
        outs.append((u.cpu().numpy(), st["iterations"], st["rel_residual"]))
        s.close()
    assert outs[0][1] == outs[1][1] and outs[0][2] == outs[1][2]
    assert np.array_equal(outs[0][0], outs[1][0])
