"""The multi-solve engine (batched solves, serving): results against the oracle's direct
solve, a solve alone vs in a mix of other solves (bitwise), graphs vs plain launches,
admission errors, and the bounded grid-barrier time-out path."""
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

ABC, NEU = wl.ABC, wl.NEUMANN


def small_random(i, n):
    return wl.random_2d_instance(i, n=n)


def odd_2d():
    n = (37, 29)
    h = 1.0 / 37
    rng = np.random.Generator(np.random.PCG64(13))
    c = 1.0 + rng.random((30, 38))
    g = (rng.standard_normal((30, 38)) + 1j * rng.standard_normal((30, 38))).astype(np.complex128)
    return wl.Workload(name="odd2d", n=n, h=h, c=c, omega=11.0, faces=(ABC,) * 4 + (NEU, NEU),
                       dt_target=0.4 * h / 2.0, mask=wl.sphere_mask(n, h, (0.5, 0.4), 0.12), g=g)


def mix():
    return [wl.gaussian_2d(n=40), odd_2d(), wl.sphere_3d(n=16), small_random(3, 45), small_random(7, 60)]


def solver(w, precision, stream, runup=0):
    return cmcg.Solver(w.n, w.h, w.c, w.omega, w.faces, mask=w.mask, order=w.order, precision=precision,
                       dt=w.dt_target, flags=cmcg.FLAG_INEXACT_RIESZ, stream=stream, runup_periods=runup)


def wrel(dz, a, b):
    return math.sqrt(float(np.sum(dz.W * np.abs(a - b) ** 2) / np.sum(dz.W * np.abs(b) ** 2)))


STREAM = None


def engine_stream():
    global STREAM
    if STREAM is None:
        STREAM = torch.cuda.Stream()
    return STREAM


def run_engine(ws, precision, tol, flags=0, runup=0):
    stream = engine_stream()
    eng = cmcg.Engine(max_slots=len(ws), stream=stream, flags=flags)
    solvers = [solver(w, precision, stream, runup) for w in ws]
    slots = [eng.submit(s, w.f, w.g, tol) for s, w in zip(solvers, ws)]
    res = eng.run_all()
    out = [res[sl] for sl in slots]
    info = eng.info()
    eng.close()
    return out, info


@pytest.mark.parametrize("precision,tol,bound", [(cmcg.MIXED, 1e-9, 1e-6), (cmcg.FP32, 1e-6, 1e-4)])
def test_batch_matches_direct(precision, tol, bound):
    ws = mix()
    out, info = run_engine(ws, precision, tol)
    assert info["graph_builds"] >= 1 and info["ticks"] >= 1
    for w, (u, st) in zip(ws, out):
        assert st["status"] == cmcg.OK, (w.name, st)
        dz = Discretization(w.n, w.h, w.c, w.omega, w.faces, w.dt_target, order=w.order, mask=w.mask)
        U = direct.solve(dz, dz.load(w.f, w.g))
        assert wrel(dz, u.cpu().numpy(), U) <= bound, (w.name, st)
        assert st["point_updates"] == st["periods"] * dz.N * dz.size


@pytest.mark.parametrize("precision", [cmcg.MIXED, cmcg.FP32])
def test_alone_equals_in_the_mix(precision):
    ws = mix()
    tol = 1e-8 if precision == cmcg.MIXED else 1e-6
    mixed, _ = run_engine(ws, precision, tol)
    for k in (0, 2):
        alone, _ = run_engine([ws[k]], precision, tol)
        assert torch.equal(alone[0][0], mixed[k][0]), ws[k].name
        assert alone[0][1]["iterations"] == mixed[k][1]["iterations"]


def test_engine_launch_shapes_agree():
    # the batched kernel's launch shape (resident blocks per SM, z-planes per 3D work item) only
    # changes how the nodes are split over blocks: the same bits for every shape
    ws = mix()[:3]
    stream = engine_stream()
    outs = []
    for shape in (None, (1, 4), (2, 32)):
        eng = cmcg.Engine(max_slots=len(ws), stream=stream, shape=shape)
        solvers = [solver(w, cmcg.FP32, stream) for w in ws]
        slots = [eng.submit(s, w.f, w.g, 1e-6) for s, w in zip(solvers, ws)]
        res = eng.run_all()
        outs.append([res[sl][0] for sl in slots])
        with pytest.raises(cmcg.CMCGError):  # a solve is active: no shape change
            s2 = solver(ws[0], cmcg.FP32, stream)
            eng.submit(s2, ws[0].f, ws[0].g, 1e-6)
            eng.set_shape(2, 8)
        eng.run_all()
        eng.close()
    for o in outs[1:]:
        assert all(torch.equal(a, b) for a, b in zip(o, outs[0]))


def test_graph_and_plain_launches_agree():
    ws = mix()[:3]
    a, _ = run_engine(ws, cmcg.MIXED, 1e-8)
    b, info = run_engine(ws, cmcg.MIXED, 1e-8, flags=cmcg.ENGINE_NO_GRAPH)
    assert info["graph_builds"] == 0
    for (ua, _), (ub, _) in zip(a, b):
        assert torch.equal(ua, ub)


def test_runup_in_the_engine():
    # Sec. 4.2.3 inside the engine (mixed precision): the zero guess sets the tolerance reference,
    # then each slot runs its ramped run-up as one unit; same fixed point, fewer CG iterations
    ws = mix()
    out0, _ = run_engine(ws, cmcg.MIXED, 1e-9)
    out1, info = run_engine(ws, cmcg.MIXED, 1e-9, runup=-1)
    for w, (u, st), (_, st0) in zip(ws, out1, out0):
        assert st["status"] == cmcg.OK and st["runup_periods"] > 0, (w.name, st)
        dz = Discretization(w.n, w.h, w.c, w.omega, w.faces, w.dt_target, order=w.order, mask=w.mask)
        U = direct.solve(dz, dz.load(w.f, w.g))
        assert wrel(dz, u.cpu().numpy(), U) <= 1e-6, (w.name, st)
        assert st["J0"] == pytest.approx(st0["J0"], rel=1e-9)
    assert sum(st["iterations"] for _, st in out1) < sum(st["iterations"] for _, st in out0)
    # a solve alone gives the same bits as in the mix
    alone, _ = run_engine([ws[2]], cmcg.MIXED, 1e-9, runup=-1)
    assert torch.equal(alone[0][0], out1[2][0])
    # FP32 slots take no run-up
    stream = engine_stream()
    eng = cmcg.Engine(max_slots=1, stream=stream)
    w = wl.gaussian_2d(n=24)
    with pytest.raises(cmcg.CMCGError) as e:
        eng.submit(solver(w, cmcg.FP32, stream, -1), w.f, None, 1e-6)
    assert e.value.code == cmcg.ERR_UNSUPPORTED
    eng.close()


def test_admission_errors():
    stream = engine_stream()
    eng = cmcg.Engine(max_slots=1, stream=stream)
    w = wl.gaussian_2d(n=24)
    s64 = cmcg.Solver(w.n, w.h, w.c, w.omega, w.faces, precision=cmcg.FP64, dt=w.dt_target, stream=stream)
    with pytest.raises(cmcg.CMCGError) as e:
        eng.submit(s64, w.f, None, 1e-6)
    assert e.value.code == cmcg.ERR_UNSUPPORTED
    s1 = solver(w, cmcg.FP32, stream)
    s2 = solver(w, cmcg.FP32, stream)
    eng.submit(s1, w.f, None, 1e-6)
    with pytest.raises(cmcg.CMCGError) as e:
        eng.submit(s1, w.f, None, 1e-6)
    assert e.value.code == cmcg.ERR_INVALID_ARG
    with pytest.raises(cmcg.CMCGError) as e:
        eng.submit(s2, w.f, None, 1e-6)
    assert e.value.code == cmcg.ERR_WORKSPACE
    eng.run_all()
    eng.close()


def test_barrier_timeout_is_reported_and_engine_recovers():
    stream = engine_stream()
    eng = cmcg.Engine(max_slots=2, stream=stream)
    assert eng.barrier_selftest(spin_limit=20000) == cmcg.ERR_DEVICE_TIMEOUT
    w = wl.gaussian_2d(n=24)
    s = solver(w, cmcg.MIXED, stream)
    eng.submit(s, w.f, None, 1e-8)
    res = eng.run_all()
    (u, st), = res.values()
    assert st["status"] == cmcg.OK
    eng.close()


def test_serving_loop_results_match_alone():
    from paper_1903_12522_gb300 import serve

    # arrivals on a simulated clock of 1 ms per tick: the admission pattern (who joins while
    # whom is running, which slot a request lands in) is the same on every run
    reqs = serve.poisson_requests(8, rate=400.0, seed=9, two_d=(24, 48), three_d=(10, 16))
    out = serve.serve(reqs, budget_bytes=int(4e9), max_slots=4, tol=1e-7, keep_results=True, stream=engine_stream(),
                      tick_s=1e-3)
    assert out["requests"] == 8 and out["status_ok"] == 8
    # requests joined while others ran, and some were admitted into slots freed by others
    assert any(r.admitted > min(q.admitted for q in reqs) and r.admitted < max(q.finished for q in reqs)
               for r in reqs)
    assert max(r.admitted for r in reqs) > min(r.finished for r in reqs)
    assert out["latency_ms"]["p50"] <= out["latency_ms"]["p99"]
    # a request solved alone gives the same field as inside the served mix
    stream = engine_stream()
    for r in reqs[:3]:
        c, f = r.build("cuda")
        eng = cmcg.Engine(max_slots=1, stream=stream)
        s = serve.make_solver(r, c, cmcg.MIXED, stream)
        slot = eng.submit(s, f, None, 1e-7)
        (u, st), = eng.run_all().values()
        eng.close()
        assert torch.equal(u.reshape(-1), r.result.reshape(-1)), r.rid


def test_default_stream_runs_without_graphs():
    ws = mix()[:2]
    stream = torch.cuda.current_stream()
    eng = cmcg.Engine(max_slots=2, stream=stream)
    solvers = [solver(w, cmcg.MIXED, stream) for w in ws]
    for s, w in zip(solvers, ws):
        eng.submit(s, w.f, w.g, 1e-8)
    res = eng.run_all()
    assert eng.info()["graph_builds"] == 0
    assert all(st["status"] == cmcg.OK for _, st in res.values())
    eng.close()


def test_refilled_slot_builds_a_new_graph_and_matches_alone():
    # A solve finishes in slot 0; its result is read, its handle destroyed and its workspace
    # released; a new solve of the same shape is admitted and lands in slot 0 (possibly with a
    # handle at the same address and the same workspace memory).  The engine must not replay
    # the graph it captured for the old solve: it builds a new one, and the new solve's field
    # equals its solve alone bit for bit.
    stream = engine_stream()
    w_long = small_random(7, 120)
    w_short = wl.gaussian_2d(n=40)
    w_new = small_random(3, 40)  # same grid as the short solve: same workspace size
    alone_new, _ = run_engine([w_new], cmcg.MIXED, 1e-8)
    eng = cmcg.Engine(max_slots=2, stream=stream)
    s_short = solver(w_short, cmcg.MIXED, stream)
    s_long = solver(w_long, cmcg.MIXED, stream)
    assert eng.submit(s_short, w_short.f, w_short.g, 1e-6) == 0
    assert eng.submit(s_long, w_long.f, w_long.g, 1e-10) == 1
    finished = []
    while 0 not in finished:
        finished = eng.tick()
        assert 1 not in finished, "the long solve must outlast the short one"
    u0, st0 = eng.result(0)
    assert st0["status"] == cmcg.OK
    s_short.close()
    del s_short
    builds = eng.info()["graph_builds"]
    assert builds >= 1
    s_new = solver(w_new, cmcg.MIXED, stream)
    assert eng.submit(s_new, w_new.f, w_new.g, 1e-8) == 0
    res = eng.run_all()
    assert eng.info()["graph_builds"] > builds
    u_new, st_new = res[0]
    assert st_new["status"] == cmcg.OK and res[1][1]["status"] == cmcg.OK
    assert torch.equal(u_new, alone_new[0][0])
    assert st_new["iterations"] == alone_new[0][1]["iterations"]
    eng.close()
