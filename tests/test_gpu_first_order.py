"""Parity of the first-order (staggered) CUDA path with the oracle (Sec. 3): the forward period
and the transposed period element by element, the dot-product test on the device, and solves
against the direct solve of the (second-order) time-discrete Helmholtz system, through both
recoveries (Eq. mix_solution and the filter of Eq. TH_FILTERED_MIXED_SOLUTION).  Tolerances:
FP64 relative L2 <= 1e-12 per period, <= 1e-9 for solves at tol 1e-12; FP32 <= 2e-5 per
period, <= 1e-4 for solves at tol 1e-6."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from oracle import direct  # noqa: E402
from oracle import first_order as ofo  # noqa: E402
from oracle.grid import Discretization  # noqa: E402
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


CASES = {
    "gauss2d_40": lambda: wl.gaussian_2d(n=40),
    "cavity2d_48": lambda: wl.square_obstacle_2d(n=48, cavity=True, wavelengths=4.0),
    "odd3d_13x11x15": odd_3d,
    "sphere3d_24": lambda: wl.sphere_3d(n=24),
    "mixed2d": mixed_2d,
}


@pytest.fixture(scope="module", params=list(CASES))
def case(request):
    w = CASES[request.param]()
    dz = Discretization(w.n, w.h, w.c, w.omega, w.faces, w.dt_target, mask=w.mask)
    return request.param, w, dz, ofo.Staggered(dz)


def solver_of(w, precision=cmcg.FP64, flags=0, **kw):
    return cmcg.Solver(w.n, w.h, w.c, w.omega, w.faces, mask=w.mask, precision=precision, dt=w.dt_target,
                       flags=cmcg.FLAG_FIRST_ORDER | flags, **kw)


def pack(p, v):
    return np.concatenate([x.ravel() for x in p] + [v.ravel()])


def unpack(s, dz):
    s = np.asarray(s).reshape(dz.dim + 1, -1)
    return [s[a].reshape(dz.shape) for a in range(dz.dim)], s[dz.dim].reshape(dz.shape)


def rand_state(st, dz, seed):
    rng = np.random.Generator(np.random.PCG64(seed))
    return [rng.standard_normal(dz.shape) * st.edge[a] for a in range(dz.dim)], rng.standard_normal(dz.shape) * dz.act


def rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def wrel(dz, a, b):
    return math.sqrt(float(np.sum(dz.W * np.abs(a - b) ** 2) / np.sum(dz.W * np.abs(b) ** 2)))


@pytest.mark.parametrize("precision,tol", [(cmcg.FP64, 1e-12), (cmcg.FP32, 2e-5)])
def test_fo_period(case, precision, tol):
    name, w, dz, st = case
    s = solver_of(w, precision)
    assert s.info["steps_per_period"] == dz.N
    p0, v0 = rand_state(st, dz, 21)
    F = dz.load(w.f, w.g)
    ref = pack(*st.period(p0, v0, F))
    out = s.fo_period(pack(p0, v0), w.f, w.g).cpu().numpy()
    assert rel(out, ref) <= tol, name
    ref_h = pack(*st.period(p0, v0, None))
    out_h = s.fo_period(pack(p0, v0)).cpu().numpy()
    assert rel(out_h, ref_h) <= tol, name


@pytest.mark.parametrize("precision,tol", [(cmcg.FP64, 1e-12), (cmcg.FP32, 2e-5)])
def test_fo_adjoint_period(case, precision, tol):
    name, w, dz, st = case
    s = solver_of(w, precision)
    y = rand_state(st, dz, 22)
    ref = pack(*st.transposed_period(*y))
    out = s.fo_adjoint_period(pack(*y)).cpu().numpy()
    assert rel(out, ref) <= tol, name


def test_fo_dot_product_on_device(case):
    name, w, dz, st = case
    s = solver_of(w)
    x = torch.as_tensor(pack(*rand_state(st, dz, 23)), device="cuda")
    y = torch.as_tensor(pack(*rand_state(st, dz, 24)), device="cuda")
    px = s.fo_period(x)
    qy = s.fo_adjoint_period(y)
    lhs, rhs = float(torch.dot(px, y)), float(torch.dot(x, qy))
    assert abs(lhs - rhs) <= 1e-12 * (abs(lhs) + abs(rhs)), name


@pytest.mark.parametrize("precision,flags,tol,bound", [(cmcg.FP64, 0, 1e-12, 5e-8),
                                                       (cmcg.FP64, cmcg.FLAG_FILTER, 1e-12, 1e-9),
                                                       (cmcg.MIXED, cmcg.FLAG_FILTER, 1e-10, 1e-8),
                                                       (cmcg.FP32, cmcg.FLAG_FILTER, 1e-6, 1e-3)])
def test_fo_solve_matches_second_order_direct(case, precision, flags, tol, bound):
    # the first-order fixed point is the second-order scheme's discrete Helmholtz solution.
    # Recovery by Eq. mix_solution reads the state at t = 0, which keeps whatever part of the
    # nearly periodic spurious modes (Sec. 3.2) the CG has not removed; the filter removes
    # them.  On the 25^3 sphere at tol 1e-12 the oracle's own first-order CG gives 1.3e-8 by
    # Eq. mix_solution and 3e-13 by the filter, hence the looser FP64 bound for the former.
    # With FP32 periods only the filter is tested: rounding excites the nearly periodic
    # spurious modes, which barely move the residual and which the recovery of Eq.
    # mix_solution (the state at t = 0) keeps (0.32 on mixed2d at rel 1.3e-4), while the
    # filter removes them.  FP32 periods make (g, d)_E noisy at the FP32 floor: the CG may stop there (NOT_CONVERGED
    # with the last iterate) before tol; the answer's accuracy is what is checked.  The floor of
    # the first-order state is higher than the second-order one's (1e-4 on mixed2d): the period
    # map fixes every divergence-free link field, a null space of dimension ~(d-1) N_p, and in
    # FP32 their divergence is rounding noise rather than zero; CMCG_MIXED removes the floor.
    name, w, dz, st = case
    U = direct.solve(dz, dz.load(w.f, w.g))
    u, stats = solver_of(w, precision, flags).solve(w.f, w.g, tol=tol)
    if precision != cmcg.FP32:
        assert stats["status"] == cmcg.OK, (name, stats)
    else:
        assert stats["status"] == cmcg.OK or (stats["status"] == cmcg.NOT_CONVERGED and
                                              stats["rel_residual"] <= 1e-3), (name, stats)
    assert stats["riesz_iterations"] == 0
    assert wrel(dz, u.cpu().numpy(), U) <= bound, (name, stats["iterations"], stats["rel_residual"])


# the oracle's CG on the 25^3 sphere takes minutes; the other cases cover 2D and 3D
@pytest.mark.parametrize("name", [k for k in CASES if k != "sphere3d_24"])
def test_fo_iterations_match_oracle(name):
    w = CASES[name]()
    dz = Discretization(w.n, w.h, w.c, w.omega, w.faces, w.dt_target, mask=w.mask)
    F = dz.load(w.f, w.g)
    ref = ofo.solve(dz, F, tol=1e-10)
    u, stats = solver_of(w).solve(w.f, w.g, tol=1e-10)
    assert abs(stats["iterations"] - ref.iterations) <= 1, (name, stats["iterations"], ref.iterations)
    assert wrel(dz, u.cpu().numpy(), ref.u) <= 1e-8
    assert stats["J0"] == pytest.approx(ref.J_history[0], rel=1e-10)


@pytest.mark.parametrize("precision,flags,tol,bound", [(cmcg.FP64, cmcg.FLAG_FILTER, 1e-12, 1e-9),
                                                       (cmcg.MIXED, cmcg.FLAG_FILTER, 1e-10, 1e-8)])
@pytest.mark.parametrize("runup", [-1, -4])
def test_fo_runup_keeps_the_fixed_point_and_saves_iterations(precision, flags, tol, bound, runup):
    # Sec. 4.2.3 on the first-order state: the ramped run-up gives the initial guess, the
    # tolerance stays referenced to the zero guess, so the answer's accuracy is unchanged
    w = wl.sphere_3d(n=24)
    dz = Discretization(w.n, w.h, w.c, w.omega, w.faces, w.dt_target, mask=w.mask)
    U = direct.solve(dz, dz.load(w.f, w.g))
    _, st0 = solver_of(w, precision, flags).solve(w.f, w.g, tol=tol)
    u1, st1 = solver_of(w, precision, flags, runup_periods=runup).solve(w.f, w.g, tol=tol)
    assert st1["status"] == cmcg.OK and st1["runup_periods"] > 0, st1
    assert wrel(dz, u1.cpu().numpy(), U) <= bound
    assert st1["iterations"] < st0["iterations"], (st0["iterations"], st1["iterations"])
    assert st1["J0"] == pytest.approx(st0["J0"], rel=1e-6)


def test_fo_unsupported_combinations():
    w = wl.gaussian_2d(n=24)
    for kw in ({"flags": cmcg.FLAG_INEXACT_RIESZ}, {"flags": cmcg.FLAG_NO_CG, "runup_periods": 2}):
        kw = dict(kw)
        flags = kw.pop("flags", 0)
        with pytest.raises(cmcg.CMCGError) as e:
            solver_of(w, flags=flags, **kw)
        assert e.value.code == cmcg.ERR_UNSUPPORTED
    lay = wl.layered_3d(n=8)
    with pytest.raises(cmcg.CMCGError) as e:
        cmcg.Solver(lay.n, lay.h, lay.c, lay.omega, lay.faces, order=4, dt=lay.dt_target, flags=cmcg.FLAG_FIRST_ORDER)
    assert e.value.code == cmcg.ERR_UNSUPPORTED
    s = solver_of(w)
    z = torch.zeros(w.num_nodes, dtype=torch.float64, device="cuda")
    with pytest.raises(cmcg.CMCGError) as e:
        s.wave_period(z, z)
    assert e.value.code == cmcg.ERR_UNSUPPORTED
    s2 = cmcg.Solver(w.n, w.h, w.c, w.omega, w.faces, dt=w.dt_target)
    with pytest.raises(cmcg.CMCGError) as e:
        s2.fo_period(torch.zeros(3 * w.num_nodes, dtype=torch.float64, device="cuda"))
    assert e.value.code == cmcg.ERR_UNSUPPORTED


def test_fo_full_size_fp32_matches_fp64_and_dot_product():
    # 257^3 sphere workload: properties that hold at any size (FP32 period within FP32 accuracy
    # of the FP64 period; FP64 transpose passes the dot-product test)
    w = wl.sphere_3d(n=256)
    gen = torch.Generator(device="cuda")
    gen.manual_seed(5)
    n4 = 4 * w.num_nodes
    x = torch.randn(n4, generator=gen, device="cuda", dtype=torch.float64)
    y = torch.randn(n4, generator=gen, device="cuda", dtype=torch.float64)
    s64 = solver_of(w, cmcg.FP64)
    p64 = s64.fo_period(x, None, w.g)
    qy = s64.fo_adjoint_period(y)
    px = s64.fo_period(x)
    # the library masks missing links and Dirichlet nodes on input and output of both maps,
    # so the identity holds for unmasked x, y as well
    lhs = float(torch.dot(px, y))
    rhs = float(torch.dot(x, qy))
    assert abs(lhs - rhs) <= 1e-11 * (abs(lhs) + abs(rhs))
    s64.close()
    del s64, px, qy
    torch.cuda.empty_cache()
    s32 = solver_of(w, cmcg.FP32)
    p32 = s32.fo_period(x, None, w.g)
    assert float(torch.linalg.vector_norm(p32 - p64) / torch.linalg.vector_norm(p64)) <= 5e-5
