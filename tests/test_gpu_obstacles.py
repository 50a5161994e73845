"""Sec. 4.2 on the GPU: plane-wave scattering off a convex square and off a semi-open square
cavity (129^2 nodes, 10 wavelengths across).  The do-nothing long-time solver converges on the
convex obstacle but stalls in the cavity, where trapped modes decay very slowly; CMCG reaches
the direct solve of the same discrete system in both.  The references are the oracle's direct
solves."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from oracle import direct  # noqa: E402
from oracle.grid import Discretization  # noqa: E402
from paper_1903_12522_gb300 import cmcg  # noqa: E402
from paper_1903_12522_gb300 import workloads as wl  # noqa: E402


@pytest.fixture(scope="module", params=[False, True], ids=["square", "cavity"])
def scatter(request):
    w = wl.square_obstacle_2d(n=128, cavity=request.param)
    dz = Discretization(w.n, w.h, w.c, w.omega, w.faces, w.dt_target, mask=w.mask)
    U = direct.solve(dz, dz.load(None, w.g))
    return request.param, w, dz, U


def wrel(dz, a, b):
    return math.sqrt(float(np.sum(dz.W * np.abs(a - b) ** 2) / np.sum(dz.W * np.abs(b) ** 2)))


def solver(w, precision, flags=0, runup=0):
    return cmcg.Solver(w.n, w.h, w.c, w.omega, w.faces, mask=w.mask, precision=precision, dt=w.dt_target,
                       flags=flags, runup_periods=runup)


def test_do_nothing_stalls_only_in_the_cavity(scatter):
    cavity, w, dz, U = scatter
    errs = []
    for ell in (50, 200):
        u, st = solver(w, cmcg.FP64, cmcg.FLAG_NO_CG, ell).solve(None, w.g, tol=1e-6)
        assert st["status"] == cmcg.OK and st["periods"] == ell
        errs.append(wrel(dz, u.cpu().numpy(), U))
    if cavity:
        # trapped modes: still far from the time-harmonic state after 200 periods
        assert errs[1] >= 0.05, errs
    else:
        assert errs[1] <= 1e-4 and errs[1] < 0.1 * errs[0], errs


@pytest.mark.parametrize("precision,flags,tol,bound", [(cmcg.FP64, 0, 1e-11, 1e-8),
                                                       (cmcg.MIXED, cmcg.FLAG_INEXACT_RIESZ, 1e-9, 1e-6)])
def test_cmcg_converges_for_both_obstacles(scatter, precision, flags, tol, bound):
    cavity, w, dz, U = scatter
    u, st = solver(w, precision, flags, runup=-1).solve(None, w.g, tol=tol)
    assert st["status"] == cmcg.OK, st
    assert wrel(dz, u.cpu().numpy(), U) <= bound, (cavity, st["iterations"])
