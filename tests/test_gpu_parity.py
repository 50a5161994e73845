"""Parity of the CUDA path (through the C ABI) with the CPU oracle, element by element.

Sizes span several thread blocks with ragged tails (41^2, 25^3, 17^3) and every boundary
type; full-size (257^3) checks compare sampled nodes with the oracle run on the node's
domain of dependence.  Tolerances: FP64 relative L2 <= 1e-12 per period and <= 1e-10 for
converged solves; FP32 stepping <= 2e-5 per period and <= 1e-4 for solves; the mixed
defect-correction solve <= 1e-6.
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from oracle import cmcg as ocmcg  # noqa: E402
from oracle import direct, wave  # noqa: E402
from oracle.grid import Discretization  # noqa: E402
from oracle.riesz import RieszSolver  # noqa: E402
from paper_1903_12522_gb300 import cmcg  # noqa: E402
from paper_1903_12522_gb300 import workloads as wl  # noqa: E402

ABC, NEU, DIR = wl.ABC, wl.NEUMANN, wl.DIRICHLET


def mixed_2d():
    n = (40, 30)
    h = 1.0 / 40
    rng = np.random.Generator(np.random.PCG64(11))
    shape = (31, 41)
    c = 1.0 + 0.8 * rng.random(shape)
    f = wl.gaussian_source(n, h, (0.3, 0.4), 0.08) * (1 + 0.5j)
    g = (rng.standard_normal(shape) + 1j * rng.standard_normal(shape)).astype(np.complex128)
    return wl.Workload(name="mixed2d", n=n, h=h, c=c, omega=9.0, faces=(ABC, DIR, NEU, ABC, NEU, NEU),
                       dt_target=0.35 * h / 1.8, f=f, g=g)


def odd_3d():
    n = (13, 11, 15)
    h = 1.0 / 15
    rng = np.random.Generator(np.random.PCG64(12))
    shape = (16, 12, 14)
    c = 1.0 + 0.5 * rng.random(shape)
    f = wl.gaussian_source(n, h, (0.4, 0.3, 0.5), 0.1).astype(np.complex128)
    return wl.Workload(name="odd3d", n=n, h=h, c=c, omega=7.0, faces=(ABC, ABC, NEU, ABC, ABC, ABC),
                       dt_target=0.3 * h / 1.5, f=f)


def odd_2d():
    n = (37, 29)
    h = 1.0 / 37
    shape = (30, 38)
    rng = np.random.Generator(np.random.PCG64(13))
    c = 1.0 + rng.random(shape)
    g = (rng.standard_normal(shape) + 1j * rng.standard_normal(shape)).astype(np.complex128)
    mask = wl.sphere_mask(n, h, (0.5, 0.4), 0.12)
    return wl.Workload(name="odd2d", n=n, h=h, c=c, omega=11.0, faces=(ABC,) * 4 + (NEU, NEU),
                       dt_target=0.4 * h / 2.0, mask=mask, g=g)


CASES = {
    "gauss2d_40": lambda: wl.gaussian_2d(n=40),
    "odd2d_37x29": odd_2d,
    "odd3d_13x11x15": odd_3d,
    "sphere3d_24": lambda: wl.sphere_3d(n=24),
    "layered3d_o4_16": lambda: wl.layered_3d(n=16),
    "mixed2d": mixed_2d,
}


def dz_of(w):
    return Discretization(w.n, w.h, w.c, w.omega, w.faces, w.dt_target, order=w.order, mask=w.mask)


def solver_of(w, precision=cmcg.FP64, **kw):
    return cmcg.Solver(w.n, w.h, w.c, w.omega, w.faces, mask=w.mask, order=w.order, precision=precision,
                       dt=w.dt_target, **kw)


def rel(a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    return float(np.linalg.norm((a - b).ravel()) / max(np.linalg.norm(b.ravel()), 1e-300))


def wrel(dz, a, b):
    return math.sqrt(float(np.sum(dz.W * np.abs(a - b) ** 2) / np.sum(dz.W * np.abs(b) ** 2)))


def rand_state(dz, seed):
    a, b = wl.random_fields(dz.shape, 2, seed)
    return a * dz.act, b * dz.act


@pytest.fixture(scope="module", params=list(CASES))
def case(request):
    w = CASES[request.param]()
    return request.param, w, dz_of(w)


def test_steps_per_period_match(case):
    name, w, dz = case
    s = solver_of(w)
    assert s.info["steps_per_period"] == dz.N
    assert abs(s.info["dt"] - dz.dt) <= 1e-15 * dz.dt
    assert bool(s.info["has_dirichlet"]) == dz.has_dirichlet


@pytest.mark.parametrize("precision,tol", [(cmcg.FP64, 1e-12), (cmcg.FP32, 2e-5)])
def test_wave_period(case, precision, tol):
    name, w, dz = case
    s = solver_of(w, precision)
    y0, v0 = rand_state(dz, 1)
    F = dz.load(w.f, w.g)
    yT, vT = wave.period(dz, y0, v0, F)
    uT, uV = s.wave_period(y0, v0, w.f, w.g)
    assert rel(uT.cpu().numpy(), yT) <= tol, name
    assert rel(uV.cpu().numpy(), vT) <= tol, name
    # homogeneous period too
    yT0, vT0 = wave.period(dz, y0, v0, None)
    uT0, uV0 = s.wave_period(y0, v0)
    assert rel(uT0.cpu().numpy(), yT0) <= tol and rel(uV0.cpu().numpy(), vT0) <= tol


@pytest.mark.parametrize("precision,tol", [(cmcg.FP64, 1e-12), (cmcg.FP32, 2e-5)])
def test_adjoint_period(case, precision, tol):
    name, w, dz = case
    s = solver_of(w, precision)
    a, b = rand_state(dz, 2)
    q0, q1 = wave.transposed_period(dz, a, b)
    g0, g1 = s.adjoint_period(a, b)
    assert rel(g0.cpu().numpy(), q0) <= tol, name
    assert rel(g1.cpu().numpy(), q1) <= tol, name


@pytest.mark.parametrize("tile", [(0, 0, 0, 2), (0, 8, 8, 2), (0, 3, 16, 2), (1, 1, 4, 2), (3, 5, 60, 2), (16, 0, 0, 3), (3, 0, 0, 3),
                                  (0, 0, 0, 4), (3, 0, 0, 4), (0, 2, 0, 4), (5, 1, 0, 4), (16, 0, 4, 3), (5, 0, 4, 3),
                                  (0, 0, 0, 5), (0, 0, 0, 6), (3, 1, 3, 6), (5, 2, 2, 6)])
@pytest.mark.parametrize("name", ["odd3d_13x11x15", "sphere3d_24"])  # the 3D 7-point cases
def test_step_scheme_variants(name, tile):
    # FP32 periods with the alternative step kernels: two steps per launch (temporal blocking,
    # scheme 2: tile[0] planes staged ahead, tile[1] planes per block, tile[2] tile height), two z-planes per thread iteration (scheme 3), operands staged by bulk copies
    # into a shared-memory ring (scheme 4: tile[0] planes per CTA, tile[1] band rows), and one
    # aligned float4 of the flat node index per thread (scheme 5), and operands staged by
    # asynchronous copies (scheme 6: tile[0] planes per CTA, tile[1] band rows, tile[2] depth);
    # schemes 5 and 6 also run forced steps
    w = CASES[name]()
    dz = dz_of(w)
    assert w.dim == 3 and w.order == 2
    s = solver_of(w, cmcg.FP32, tile=tile)
    y0, v0 = rand_state(dz, 6)
    yT, vT = wave.period(dz, y0, v0, None)
    uT, uV = s.wave_period(y0, v0)
    assert rel(uT.cpu().numpy(), yT) <= 2e-5 and rel(uV.cpu().numpy(), vT) <= 2e-5
    q0, q1 = wave.transposed_period(dz, y0, v0)
    g0, g1 = s.adjoint_period(y0, v0)
    assert rel(g0.cpu().numpy(), q0) <= 2e-5 and rel(g1.cpu().numpy(), q1) <= 2e-5
    if tile[3] in (3, 5, 6):  # forced steps too (on the sphere the source sits on the faces only,
        # so the z-pair kernels skip it inside the interior columns)
        yF, vF = wave.period(dz, y0, v0, dz.load(w.f, w.g))
        uF, uVF = s.wave_period(y0, v0, w.f, w.g)
        assert rel(uF.cpu().numpy(), yF) <= 2e-5 and rel(uVF.cpu().numpy(), vF) <= 2e-5


@pytest.mark.parametrize("tile", [(0, 0, 0, 1), (3, 0, 0, 1), (0, 0, 0, 3), (3, 0, 0, 3), (5, 0, 0, 0)])
def test_step13_variants(tile):
    # the 4th-order (13-point) step: one z-plane per loop trip (scheme 1) and two (scheme 3,
    # the default); tile[0] z-planes per block gives ragged chunks on the 17^3 grid.  FP32 and
    # FP64, forced and homogeneous periods, and the adjoint
    w = CASES["layered3d_o4_16"]()
    dz = dz_of(w)
    assert w.order == 4 and w.dim == 3
    y0, v0 = rand_state(dz, 8)
    F = dz.load(w.f, w.g)
    yF, vF = wave.period(dz, y0, v0, F)
    q0, q1 = wave.transposed_period(dz, y0, v0)
    for precision, tol in ((cmcg.FP64, 1e-12), (cmcg.FP32, 2e-5)):
        s = solver_of(w, precision, tile=tile)
        uF, uVF = s.wave_period(y0, v0, w.f, w.g)
        assert rel(uF.cpu().numpy(), yF) <= tol and rel(uVF.cpu().numpy(), vF) <= tol, (tile, precision)
        g0, g1 = s.adjoint_period(y0, v0)
        assert rel(g0.cpu().numpy(), q0) <= tol and rel(g1.cpu().numpy(), q1) <= tol, (tile, precision)


@pytest.mark.parametrize("name", ["gauss2d_40", "odd2d_37x29", "mixed2d"])
def test_vector_step_2d(name):
    # the vector-form step (scheme 5) on 2D 5-point grids: forced and homogeneous FP32 periods
    # and the adjoint period against the oracle
    w = CASES[name]()
    dz = dz_of(w)
    s = solver_of(w, cmcg.FP32, tile=(0, 0, 0, 5))
    y0, v0 = rand_state(dz, 8)
    for F, f, g in ((dz.load(w.f, w.g), w.f, w.g), (None, None, None)):
        yT, vT = wave.period(dz, y0, v0, F)
        uT, uV = s.wave_period(y0, v0, f, g)
        assert rel(uT.cpu().numpy(), yT) <= 2e-5 and rel(uV.cpu().numpy(), vT) <= 2e-5, name
    q0, q1 = wave.transposed_period(dz, y0, v0)
    g0, g1 = s.adjoint_period(y0, v0)
    assert rel(g0.cpu().numpy(), q0) <= 2e-5 and rel(g1.cpu().numpy(), q1) <= 2e-5, name


def test_adjoint_dot_product_on_device(case):
    name, w, dz = case
    s = solver_of(w)
    x0, x1 = rand_state(dz, 3)
    y0, y1 = rand_state(dz, 4)
    p0, p1 = [t.cpu().numpy() for t in s.wave_period(x0, x1)]
    q0, q1 = [t.cpu().numpy() for t in s.adjoint_period(y0, y1)]
    lhs = np.sum(p0 * y0) + np.sum(p1 * y1)
    rhs = np.sum(x0 * q0) + np.sum(x1 * q1)
    scale = math.sqrt(np.sum(p0 ** 2) + np.sum(p1 ** 2)) * math.sqrt(np.sum(y0 ** 2) + np.sum(y1 ** 2))
    assert abs(lhs - rhs) <= 1e-13 * scale


def test_riesz(case):
    name, w, dz = case
    s = solver_of(w, riesz_tol=1e-13)
    rhs = wl.random_fields(dz.shape, 1, 5)[0] * dz.act
    ref = RieszSolver(dz).solve(rhs)
    got, code = s.riesz(rhs)
    assert code == cmcg.OK
    assert rel(got.cpu().numpy(), ref) <= 1e-10, name


@pytest.mark.parametrize("precision,tol,bound", [(cmcg.FP64, 1e-13, 1e-10), (cmcg.FP32, 1e-6, 1e-4),
                                                 (cmcg.MIXED, 1e-8, 1e-6)])
def test_solve_matches_direct(case, precision, tol, bound):
    name, w, dz = case
    s = solver_of(w, precision)
    U = direct.solve(dz, dz.load(w.f, w.g))
    u, st = s.solve(w.f, w.g, tol=tol)
    assert st["status"] == cmcg.OK, st
    assert wrel(dz, u.cpu().numpy(), U) <= bound, (name, st)
    assert st["point_updates"] == st["periods"] * dz.N * dz.size
    if not dz.has_dirichlet:
        # Im lambda vanishes up to the solve's accuracy relative to the field's size
        assert abs(st["lambda_im"]) <= bound * max(abs(st["lambda_re"]), float(np.abs(U).max()))


@pytest.mark.parametrize("precision,tol,bound", [(cmcg.FP64, 1e-12, 5e-9), (cmcg.FP32, 1e-6, 1e-4),
                                                 (cmcg.MIXED, 1e-9, 1e-6)])
def test_inexact_riesz_solve_matches_direct(case, precision, tol, bound):
    # one V-cycle as the Riesz map inside flexible CG: same fixed point as the exact map; the
    # recursively updated residual limits the attainable FP64 accuracy to a few 1e-9
    name, w, dz = case
    s = solver_of(w, precision, flags=cmcg.FLAG_INEXACT_RIESZ)
    U = direct.solve(dz, dz.load(w.f, w.g))
    u, st = s.solve(w.f, w.g, tol=tol)
    assert st["status"] == cmcg.OK, st
    assert wrel(dz, u.cpu().numpy(), U) <= bound, (name, st)
    assert st["riesz_iterations"] >= st["iterations"]


@pytest.mark.parametrize("runup", [-1, -4])
@pytest.mark.parametrize("precision,flags,tol,bound", [(cmcg.FP64, 0, 1e-12, 1e-9),
                                                       (cmcg.MIXED, cmcg.FLAG_INEXACT_RIESZ, 1e-9, 1e-6)])
def test_runup_keeps_the_fixed_point_and_saves_iterations(precision, flags, tol, bound, runup):
    # Sec. 4.2.3: a run-up from rest with ramped sources gives the initial guess; the tolerance
    # refers to the zero-guess residual, so the answer's accuracy is unchanged
    w = wl.sphere_3d(n=24)
    dz = dz_of(w)
    U = direct.solve(dz, dz.load(w.f, w.g))
    _, st0 = solver_of(w, precision, flags=flags).solve(w.f, w.g, tol=tol)
    u1, st1 = solver_of(w, precision, flags=flags, runup_periods=runup).solve(w.f, w.g, tol=tol)
    assert st1["status"] == cmcg.OK and st1["runup_periods"] > 0
    # -k: the periods waves at c_min need to cross the domain's diagonal k times
    diam = w.h * math.sqrt(sum(m * m for m in w.n))
    assert st1["runup_periods"] == max(1, math.ceil(-runup * diam * w.omega / (2 * math.pi * 0.7) - 1e-9))
    assert wrel(dz, u1.cpu().numpy(), U) <= bound
    assert st1["iterations"] < st0["iterations"], (st0["iterations"], st1["iterations"])


@pytest.mark.parametrize("precision,tol,bound", [(cmcg.FP64, 1e-13, 1e-10), (cmcg.MIXED, 1e-9, 1e-6)])
def test_filter_recovery_matches_direct(case, precision, tol, bound):
    # Sec. 2.2: the fundamental-frequency filter over one forced period gives U without the
    # compatibility-condition shift
    name, w, dz = case
    s = solver_of(w, precision, flags=cmcg.FLAG_FILTER)
    U = direct.solve(dz, dz.load(w.f, w.g))
    u, st = s.solve(w.f, w.g, tol=tol)
    assert st["status"] == cmcg.OK and st["lambda_re"] == 0.0
    assert wrel(dz, u.cpu().numpy(), U) <= bound, name


@pytest.mark.parametrize("flags", [0, cmcg.FLAG_FILTER])
def test_pure_neumann_after_runup(flags):
    # Sec. 2.2 and 3.5: pure Neumann box (k = pi/4); from a run-up the minimiser grows
    # linearly (eta t).  Plain recovery removes the constant with lambda; the filter removes
    # the rest and fixes the constant by the discrete form of Eq. cc_neumann_eta
    w = wl.neumann_box_2d(40)
    dz = dz_of(w)
    F = dz.load(w.f, None)
    U = direct.solve(dz, F)
    u, st = solver_of(w, cmcg.FP64, flags=flags, runup_periods=2).solve(w.f, None, tol=1e-12)
    assert st["status"] == cmcg.OK and st["runup_periods"] == 2
    assert abs(complex(st["lambda_re"], st["lambda_im"])) > 1e-2
    assert wrel(dz, u.cpu().numpy(), U) <= 1e-8


@pytest.mark.parametrize("precision,bound", [(cmcg.FP64, 1e-11), (cmcg.FP32, 1e-4)])
def test_do_nothing_matches_oracle_long_time(case, precision, bound):
    # Sec. 4.2 (Eq. AP_SOLUTION): l = 3 periods of the forced wave equation from rest with the
    # ramped sources of Sec. 4.2.3, recovered as in step (6); no CG
    name, w, dz = case
    F = dz.load(w.f, w.g)
    y, v = wave.long_time(dz, F, 3)
    ref = ocmcg.asymptotic(dz, y, v, F)
    s = solver_of(w, precision, flags=cmcg.FLAG_NO_CG, runup_periods=3)
    u, st = s.solve(w.f, w.g, tol=1e-6)
    assert st["status"] == cmcg.OK and st["iterations"] == 0 and st["runup_periods"] == 3
    assert st["periods"] == 3 and st["point_updates"] == 3 * dz.N * dz.size
    assert wrel(dz, u.cpu().numpy(), ref) <= bound, name


def test_fp64_iterations_and_shift_match_oracle(case):
    name, w, dz = case
    s = solver_of(w)
    F = dz.load(w.f, w.g)
    ref = ocmcg.solve(dz, F, tol=1e-10)
    u, st = s.solve(w.f, w.g, tol=1e-10)
    assert abs(st["iterations"] - ref.iterations) <= 2, (st["iterations"], ref.iterations)
    assert abs(st["lambda_re"] - ref.lam.real) <= 1e-8 * max(abs(ref.lam), 1e-12)
    assert abs(st["J0"] - ref.J_history[0]) <= 1e-10 * ref.J_history[0]
    # the residual history (Step 5.8's quantity per iteration) follows the oracle's
    hist = s.history()
    assert len(hist) == st["iterations"] + 1 and hist[0] == pytest.approx(1.0, rel=1e-12)
    assert hist[-1] == pytest.approx(st["rel_residual"], rel=1e-12) and hist[-1] <= 1e-10
    k = min(10, len(hist), len(ref.residual_history))  # the early iterations, before rounding drifts
    assert np.allclose(hist[:k], ref.residual_history[:k], rtol=1e-6, atol=0), name


def test_l2_resident_kappa_changes_nothing_but_the_cache():
    # CMCG_FLAG_L2_KAPPA only sets an L2 access policy on kappa: the same bits, and a handle
    # created and destroyed with it leaves the next solve unchanged
    w = wl.sphere_3d(n=24)
    stream = torch.cuda.Stream()
    base = solver_of(w, cmcg.MIXED, flags=cmcg.FLAG_INEXACT_RIESZ, stream=stream).solve(w.f, w.g, tol=1e-9)
    s = solver_of(w, cmcg.MIXED, flags=cmcg.FLAG_INEXACT_RIESZ | cmcg.FLAG_L2_KAPPA, stream=stream)
    l2 = s.solve(w.f, w.g, tol=1e-9)
    s.close()
    after = solver_of(w, cmcg.MIXED, flags=cmcg.FLAG_INEXACT_RIESZ, stream=stream).solve(w.f, w.g, tol=1e-9)
    assert torch.equal(base[0], l2[0]) and torch.equal(base[0], after[0])
    assert base[1]["iterations"] == l2[1]["iterations"]


@pytest.mark.parametrize("precision,tol", [(cmcg.FP64, 1e-9), (cmcg.MIXED, 1e-9), (cmcg.FP32, 1e-6)])
def test_graph_replayed_iterations_match_plain_launches(precision, tol):
    # on its own stream a solve replays each flexible-CG iteration as a captured CUDA graph; on
    # the legacy default stream it launches the kernels one by one: same bits, same counts
    w = wl.sphere_3d(n=16)
    out = {}
    for name, stream in (("graph", torch.cuda.Stream()), ("plain", torch.cuda.default_stream())):
        s = solver_of(w, precision, flags=cmcg.FLAG_INEXACT_RIESZ, stream=stream)
        out[name] = s.solve(w.f, w.g, tol=tol)
    (ug, sg), (up, sp) = out["graph"], out["plain"]
    assert torch.equal(ug, up)
    # the history of a mixed solve ends at the FP64 residual it stopped on
    assert len(s.history()) >= 1 and s.history()[-1] == pytest.approx(sp["rel_residual"], rel=1e-12)
    for k in ("iterations", "periods", "riesz_iterations", "kernel_launches", "outer_iterations"):
        assert sg[k] == sp[k], (k, sg[k], sp[k])
    assert sp["graph_replays"] == 0
    assert 0 < sg["graph_replays"] < sg["iterations"] + 1


@pytest.mark.parametrize("precision", [cmcg.FP64, cmcg.MIXED])
def test_step_timing_inside_replayed_graphs(precision):
    # with step timing on, the event records are nodes of the captured iteration: the step
    # kernels' device time and launch count come out as with plain launches, and the
    # iterations are still replayed
    w = wl.sphere_3d(n=24)
    flags = cmcg.FLAG_INEXACT_RIESZ | cmcg.FLAG_TIMING
    out = {}
    for name, stream in (("graph", torch.cuda.Stream()), ("plain", torch.cuda.default_stream())):
        s = solver_of(w, precision, flags=flags, stream=stream)
        out[name] = s.solve(w.f, w.g, tol=1e-9)
    (ug, sg), (up, sp) = out["graph"], out["plain"]
    assert torch.equal(ug, up)
    # the history of a mixed solve ends at the FP64 residual it stopped on
    assert len(s.history()) >= 1 and s.history()[-1] == pytest.approx(sp["rel_residual"], rel=1e-12)
    assert sg["graph_replays"] >= sg["iterations"] - 2 > 0, (sg["graph_replays"], sg["iterations"])
    assert sp["graph_replays"] == 0
    for k in ("step_launches_fp32", "step_launches_fp64", "kernel_launches", "periods"):
        assert sg[k] == sp[k], (k, sg[k], sp[k])
    key = "step_seconds_fp64" if precision == cmcg.FP64 else "step_seconds_fp32"
    n_key = key.replace("seconds", "launches")
    assert sg[n_key] > 0
    per_g, per_p = sg[key] / sg[n_key], sp[key] / sp[n_key]
    assert 0.25 * per_p < per_g < 4 * per_p, (per_g, per_p)


@pytest.mark.parametrize("name", ["sphere3d_24", "gauss2d_40"])
@pytest.mark.parametrize("precision,flags,tol,bound", [(cmcg.FP64, 0, 1e-13, 1e-10),
                                                       (cmcg.MIXED, cmcg.FLAG_INEXACT_RIESZ, 1e-9, 1e-6)])
def test_warm_start_resumes_a_solve(name, precision, flags, tol, bound):
    # checkpoint / resume: a solve stopped early, then continued from its output field
    # (cmcg_solve_warm), reaches the same accuracy in fewer iterations than a cold solve; a
    # start at the exact discrete solution needs at most a couple of iterations (its periodic
    # state is the fixed point up to the direct solve's rounding; on an ABC-only box the
    # constant lambda drops out of the periodicity misfit)
    w = CASES[name]()
    dz = dz_of(w)
    s = solver_of(w, precision, flags=flags)
    U = direct.solve(dz, dz.load(w.f, w.g))
    u1, st1 = s.solve(w.f, w.g, tol=1e-3)
    assert st1["status"] == cmcg.OK and wrel(dz, u1.cpu().numpy(), U) > bound
    u2, st2 = s.solve(w.f, w.g, tol=tol, u0=u1)
    assert st2["status"] == cmcg.OK, st2
    assert wrel(dz, u2.cpu().numpy(), U) <= bound, st2
    u3, st3 = s.solve(w.f, w.g, tol=tol)
    assert st3["status"] == cmcg.OK and st2["iterations"] < st3["iterations"], (st2, st3)
    assert st2["runup_periods"] == 0
    u4, st4 = s.solve(w.f, w.g, tol=tol, u0=U)
    assert st4["status"] == cmcg.OK and st4["iterations"] <= 2, st4
    assert wrel(dz, u4.cpu().numpy(), U) <= bound


@pytest.mark.parametrize("precision,tol,bound", [(cmcg.FP64, 1e-13, 1e-10), (cmcg.MIXED, 1e-10, 1e-6)])
def test_paper_example_sec4_1_on_the_gpu(precision, tol, bound):
    # the printed example of Sec. 4.1 (tests/golden/sec4_1_semidiscrete_example.txt): u = e^{ikx},
    # omega = k = 6 pi, on the unit square (256 x 256 intervals) with absorbing x-faces (the
    # exact datum at x = 0) and Neumann y-faces, where it stays constant in y.  The GPU solve matches the direct solve, and its distance to the printed
    # solution is the discretisation error the oracle has.
    import os
    fx = {}
    for line in open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden",
                                  "sec4_1_semidiscrete_example.txt")):
        line = line.split("#", 1)[0].strip()
        if line:
            key, value = (x.strip() for x in line.split("=", 1))
            fx[key] = value
    k = float(fx["k_over_pi"]) * math.pi
    m = 256
    n, h = (m, m), 1.0 / m
    faces = (ABC, ABC, NEU, NEU, NEU, NEU)
    g = wl.plane_wave_boundary_datum(n, h, k, 1.0, (1.0, 0.0), faces)
    w = wl.Workload(name="sec4_1_square", n=n, h=h, c=np.ones((m + 1, m + 1)), omega=k, faces=faces,
                    dt_target=0.4 * h, g=g)
    dz = dz_of(w)
    U = direct.solve(dz, dz.load(None, g))
    s = solver_of(w, precision, flags=cmcg.FLAG_INEXACT_RIESZ if precision == cmcg.MIXED else 0)
    u, st = s.solve(None, g, tol=tol)
    assert st["status"] == cmcg.OK, st
    ug = u.cpu().numpy()
    assert wrel(dz, ug, U) <= bound, st
    exact = np.exp(1j * k * wl.coords(n, h)[0]) * np.ones(dz.shape)
    e_gpu, e_oracle = wrel(dz, ug, exact), wrel(dz, U, exact)
    assert abs(e_gpu - e_oracle) <= 1e-3 * e_oracle + bound and e_oracle < 3e-3, (e_gpu, e_oracle)


def test_solve_host_matches_device():
    w = wl.gaussian_2d(n=48)
    s = solver_of(w, flags=cmcg.FLAG_HOST_IO)
    u_dev, st = s.solve(w.f, None, tol=1e-10)
    u_host = np.empty(w.shape, dtype=np.complex128)
    st2 = cmcg.Stats()
    code = cmcg.cmcg_solve_host(s.handle, np.ascontiguousarray(w.f), None, 1e-10, u_host, st2)
    assert code == cmcg.OK
    assert rel(u_host, u_dev.cpu().numpy()) <= 1e-12
    assert st2.iterations == st["iterations"]


def test_deterministic():
    w = wl.sphere_3d(n=16)
    s = solver_of(w)
    u1, _ = s.solve(w.f, w.g, tol=1e-8)
    u2, _ = s.solve(w.f, w.g, tol=1e-8)
    assert torch.equal(u1, u2)


def test_zero_source_gives_zero():
    w = wl.gaussian_2d(n=24)
    s = solver_of(w)
    u, st = s.solve(None, None, tol=1e-6)
    assert st["status"] == cmcg.OK and st["iterations"] == 0
    assert float(u.abs().max()) == 0.0


def test_not_converged_returns_last_iterate():
    w = wl.gaussian_2d(n=24)
    s = solver_of(w, max_iter=3)
    u, st = s.solve(w.f, None, tol=1e-12)
    assert st["status"] == cmcg.NOT_CONVERGED and st["iterations"] == 3
    assert 0 < st["rel_residual"] < 1 and float(u.abs().max()) > 0


def tiny(n, faces, seed):
    h = 1.0 / max(n)
    shape = tuple(m + 1 for m in reversed(n))
    rng = np.random.Generator(np.random.PCG64(seed))
    c = 1.0 + 0.3 * rng.random(shape)
    f = (rng.standard_normal(shape) + 1j * rng.standard_normal(shape)).astype(np.complex128)
    return wl.Workload(name=f"tiny{n}", n=n, h=h, c=c, omega=2.5, faces=faces, dt_target=0.2 * h, f=f)


@pytest.mark.parametrize("n,faces", [((2, 2), (ABC,) * 4 + (NEU, NEU)), ((3, 2), (ABC, DIR, NEU, ABC, NEU, NEU)),
                                     ((2, 3, 2), (ABC,) * 6), ((2, 2, 3), (ABC, NEU, DIR, ABC, NEU, ABC))])
def test_smallest_grids(n, faces):
    # the smallest grids the ABI accepts (2 intervals per axis, 3 nodes): every node is a
    # boundary node, the multigrid has one level, and the step kernels' mirrors meet
    w = tiny(n, faces, 31)
    dz = dz_of(w)
    y0, v0 = rand_state(dz, 32)
    F = dz.load(w.f, None)
    yT, vT = wave.period(dz, y0, v0, F)
    for precision, tol in ((cmcg.FP64, 1e-12), (cmcg.FP32, 2e-5)):
        uT, uV = solver_of(w, precision).wave_period(y0, v0, w.f, None)
        assert rel(uT.cpu().numpy(), yT) <= tol and rel(uV.cpu().numpy(), vT) <= tol, (n, precision)
    U = direct.solve(dz, F)
    for precision, flags, tol, bound in ((cmcg.FP64, 0, 1e-12, 1e-9),
                                         (cmcg.MIXED, cmcg.FLAG_INEXACT_RIESZ, 1e-10, 1e-7)):
        u, st = solver_of(w, precision, flags=flags).solve(w.f, None, tol=tol)
        assert st["status"] == cmcg.OK, (n, st)
        assert wrel(dz, u.cpu().numpy(), U) <= bound, (n, precision)


def test_invalid_arguments():
    w = wl.gaussian_2d(n=16)
    with pytest.raises(cmcg.CMCGError) as e:
        cmcg.Solver(w.n, w.h, w.c, w.omega, w.faces, dt=2.0 * w.h)
    assert e.value.code == cmcg.ERR_CFL
    with pytest.raises(cmcg.CMCGError) as e:
        cmcg.Solver(w.n, w.h, -w.c, w.omega, w.faces, dt=w.dt_target)
    assert e.value.code == cmcg.ERR_INVALID_ARG
    w3 = wl.sphere_3d(n=8)
    with pytest.raises(cmcg.CMCGError) as e:
        cmcg.Solver(w3.n, w3.h, w3.c, w3.omega, w3.faces, mask=w3.mask, order=4, dt=0.2 * w3.h)
    assert e.value.code == cmcg.ERR_UNSUPPORTED
    # workspace too small
    g = cmcg.make_grid(w.n, w.h)
    o = cmcg.make_options(dt=w.dt_target)
    need = cmcg.cmcg_workspace_size(g, o)
    ws = torch.empty(need - 1024, dtype=torch.uint8, device="cuda")
    c = torch.as_tensor(w.c.ravel(), device="cuda")
    bc = cmcg.BC()
    with pytest.raises(cmcg.CMCGError) as e:
        cmcg.cmcg_create(g, c, w.omega, bc, o, ws, torch.cuda.current_stream().cuda_stream)
    assert e.value.code == cmcg.ERR_WORKSPACE


# ---------------------------------------------------------------------------------------
# Full size (257^3 sphere workload, the benchmark's configuration): sampled nodes against the
# oracle run on each node's domain of dependence (N + 2 nodes in every direction).
def crop(w, center, margin):
    lo, hi = [], []
    for a in range(3):
        lo.append(max(0, center[a] - margin))
        hi.append(min(w.n[a], center[a] + margin))
    sl = tuple(slice(lo[a], hi[a] + 1) for a in reversed(range(3)))
    faces = []
    for a in range(3):
        faces.append(w.faces[2 * a] if lo[a] == 0 else NEU)
        faces.append(w.faces[2 * a + 1] if hi[a] == w.n[a] else NEU)
    n = tuple(hi[a] - lo[a] for a in range(3))
    sub = wl.Workload(name="crop", n=n, h=w.h, c=w.c[sl], omega=w.omega, faces=tuple(faces),
                      dt_target=w.dt_target, order=w.order,
                      mask=None if w.mask is None else w.mask[sl],
                      f=None if w.f is None else w.f[sl], g=None if w.g is None else w.g[sl])
    local = tuple(center[a] - lo[a] for a in reversed(range(3)))
    return sub, sl, local


@pytest.fixture(scope="module")
def full_size():
    w = wl.sphere_3d(n=256)
    y0, v0 = wl.random_fields(w.shape, 2, 21)
    act = 1.0 - (w.mask.astype(np.float64))
    return w, y0 * act, v0 * act


@pytest.mark.parametrize("precision,tol,tile", [(cmcg.FP64, 1e-11, None), (cmcg.FP32, 1e-4, None),
                                               (cmcg.FP32, 1e-4, (0, 0, 0, 2)), (cmcg.FP32, 1e-4, (16, 0, 0, 3)),
                                               (cmcg.FP32, 1e-4, (0, 0, 0, 4)), (cmcg.FP32, 1e-4, (0, 0, 0, 5)),
                                               (cmcg.FP32, 1e-4, (0, 0, 0, 6))])
def test_full_size_period_sampled(full_size, precision, tol, tile):
    w, y0, v0 = full_size
    s = solver_of(w, precision, tile=tile)
    if tile is not None and tile[3] not in (5, 6):  # schemes 2-4 run homogeneous steps only: no source here
        uT, vT = [t.cpu().numpy() for t in s.wave_period(y0, v0, None, None)]
    else:
        uT, vT = [t.cpu().numpy() for t in s.wave_period(y0, v0, None, w.g)]
    N = s.info["steps_per_period"]
    samples = [(0, 0, 0), (128, 128, 103), (256, 40, 200), (7, 250, 128), (140, 131, 129)]
    for cidx in samples:
        sub, sl, local = crop(w, cidx, N + 3)
        dz = dz_of(sub)
        assert dz.N == N
        yT, vTo = wave.period(dz, y0[sl], v0[sl],
                              None if tile is not None and tile[3] not in (5, 6) else dz.load(sub.f, sub.g))
        scale = max(np.abs(yT).max(), 1e-30)
        assert abs(uT[sl][local] - yT[local]) <= tol * scale, (cidx, uT[sl][local], yT[local])
        scale_v = max(np.abs(vTo).max(), 1e-30)
        assert abs(vT[sl][local] - vTo[local]) <= tol * scale_v, cidx


@pytest.mark.parametrize("tile", [(0, 0, 0, 2), (1, 8, 12, 2), (3, 40, 0, 2), (0, 0, 0, 3), (0, 0, 0, 4), (16, 0, 4, 3), (0, 0, 0, 5),
                                  (0, 0, 0, 6), (0, 0, 3, 6)])
def test_full_size_step_kernels_agree(full_size, tile):
    # the two-step, z-pair, bulk-copy and vector-form kernels evaluate the single-step kernel's
    # expression in the same order; their FP32 periods agree with it to rounding
    w, y0, v0 = full_size
    ref = [t.reshape(-1) for t in solver_of(w, cmcg.FP32, tile=(0, 0, 0, 1)).wave_period(y0, v0)]
    out = [t.reshape(-1) for t in solver_of(w, cmcg.FP32, tile=tile).wave_period(y0, v0)]
    adj_ref = [t.reshape(-1) for t in solver_of(w, cmcg.FP32, tile=(0, 0, 0, 1)).adjoint_period(y0, v0)]
    adj = [t.reshape(-1) for t in solver_of(w, cmcg.FP32, tile=tile).adjoint_period(y0, v0)]
    for a, b in zip(out + adj, ref + adj_ref):
        assert float(torch.linalg.vector_norm(a - b) / torch.linalg.vector_norm(b)) <= 1e-6
    print("bitwise equal:", all(torch.equal(a, b) for a, b in zip(out + adj, ref + adj_ref)))


def test_bulk_wait_times_out_and_context_survives():
    # the bulk-copy kernel's mbarrier waits are bounded: a wait on a phase that nothing
    # completes runs out and reports a time-out; the context stays usable afterwards
    assert cmcg.cmcg_bulk_wait_selftest(2000) == cmcg.ERR_DEVICE_TIMEOUT
    w = wl.sphere_3d(n=16)
    dz = dz_of(w)
    y0, v0 = rand_state(dz, 9)
    yT, _ = wave.period(dz, y0, v0, None)
    uT, _ = solver_of(w, cmcg.FP32, tile=(0, 0, 0, 4)).wave_period(y0, v0)
    assert rel(uT.cpu().numpy(), yT) <= 2e-5


def test_full_size_adjoint_dot(full_size):
    w, y0, v0 = full_size
    s = solver_of(w)
    a, b = wl.random_fields(w.shape, 2, 22)
    act = 1.0 - w.mask.astype(np.float64)
    a, b = a * act, b * act
    p0, p1 = [t.cpu().numpy() for t in s.wave_period(y0, v0)]
    q0, q1 = [t.cpu().numpy() for t in s.adjoint_period(a, b)]
    lhs = np.sum(p0 * a) + np.sum(p1 * b)
    rhs = np.sum(y0 * q0) + np.sum(v0 * q1)
    scale = math.sqrt(np.sum(p0 ** 2) + np.sum(p1 ** 2)) * math.sqrt(np.sum(a ** 2) + np.sum(b ** 2))
    assert abs(lhs - rhs) <= 1e-12 * scale
