"""The serving loop's host logic without a GPU.  The engine and the solvers are replaced by
fakes that finish each request a fixed number of ticks after its admission, so the test
checks what serve.serve itself decides: admission in arrival order by workspace bytes
(cmcg_workspace_size, a host call) and free slots, never above the memory budget or the slot
count, requests joining between ticks while others run (continuous batching), rejection of a
request that could never fit, and the latency bookkeeping."""
import os

import pytest

from paper_1903_12522_gb300 import cmcg, serve

pytestmark = pytest.mark.timeout(120)  # a serving loop that never ends fails instead of hanging


@pytest.fixture(scope="module", autouse=True)
def lib():
    if not os.path.exists(cmcg.LIB_PATH):
        from paper_1903_12522_gb300 import build

        build.build()
    return cmcg.load()


def ticks_for(req):
    return 2 + req.n % 5  # deterministic, uneven solve lengths


class FakeSolver:
    def __init__(self, req):
        self.req = req
        self.closed = False

    def close(self):
        self.closed = True


class FakeEngine:
    last = None

    def __init__(self, max_slots, stream=None, shape=None):
        self.max_slots = max_slots
        self.stream = stream if stream is not None else object()
        self.running = {}  # slot -> [solver, ticks left, bytes, admission tick]
        self.ticks = 0
        self.next_slot = 0
        self.peak_slots = 0
        self.peak_bytes = 0
        self.mixed_ticks = 0  # ticks whose running set was admitted at different ticks
        self.results = {}
        FakeEngine.last = self

    def submit(self, s, f, g, tol):
        slot = self.next_slot
        self.next_slot += 1
        nb = serve.workspace_bytes(s.req, cmcg.MIXED)
        self.running[slot] = [s, ticks_for(s.req), nb, self.ticks]
        return slot

    def tick(self):
        self.peak_slots = max(self.peak_slots, len(self.running))
        self.peak_bytes = max(self.peak_bytes, sum(r[2] for r in self.running.values()))
        if len({r[3] for r in self.running.values()}) > 1:
            self.mixed_ticks += 1
        self.ticks += 1
        done = []
        for slot, r in list(self.running.items()):
            r[1] -= 1
            if r[1] == 0:
                done.append(slot)
                self.results[slot] = r[0].req
                del self.running[slot]
        return done

    def result(self, slot):
        req = self.results.pop(slot)
        return None, {"status": cmcg.OK, "point_updates": req.n ** req.dim}

    def info(self):
        return {"ticks": self.ticks, "graph_builds": 0}

    def close(self):
        pass


@pytest.fixture
def fakes(monkeypatch):
    monkeypatch.setattr(cmcg, "Engine", FakeEngine)
    monkeypatch.setattr(serve, "make_solver", lambda req, c, precision, stream, runup=0: FakeSolver(req))
    monkeypatch.setattr(serve.Request, "build", lambda self, device: (None, None))


def test_admission_respects_budget_and_slots(fakes):
    reqs = serve.poisson_requests(30, rate=2000.0, seed=3, two_d=(64, 256), three_d=(16, 48))
    sizes = [serve.workspace_bytes(r, cmcg.MIXED) for r in reqs]
    budget = 3 * max(sizes)  # only a few fit at once
    # a simulated clock of 1 ms per tick: the admission pattern does not depend on host speed
    out = serve.serve(reqs, budget_bytes=budget, max_slots=4, device="cpu", tick_s=1e-3)
    eng = FakeEngine.last
    assert out["requests"] == 30 and out["status_ok"] == 30 and out["rejected"] == 0
    assert eng.peak_slots <= 4
    assert eng.peak_bytes <= budget
    assert eng.mixed_ticks > 0  # requests joined while others ran
    for r in reqs:
        assert r.arrival <= r.admitted <= r.finished
    assert out["latency_ms"]["p50"] <= out["latency_ms"]["p99"]
    assert out["ticks"] == eng.ticks


def test_first_fit_lets_a_small_request_pass_a_large_one(fakes):
    # in arrival order: a large request that does not fit next to the running one, then a
    # small one that does; the small one is admitted first
    reqs = serve.poisson_requests(3, rate=1e6, seed=1, two_d=(64, 64), three_d=(64, 64), frac_2d=1.0)
    big = serve.Request(1, reqs[1].arrival, 2, 400, 12.0, (0.5, 0.5), 7)
    small = serve.Request(2, reqs[2].arrival, 2, 64, 12.0, (0.5, 0.5), 8)
    first = serve.Request(0, reqs[0].arrival, 2, 300, 12.0, (0.5, 0.5), 6)
    b_first, b_big, b_small = (serve.workspace_bytes(r, cmcg.MIXED) for r in (first, big, small))
    budget = b_first + max(b_small, b_big - 1)
    assert b_first + b_big > budget >= b_first + b_small and b_big <= budget
    out = serve.serve([first, big, small], budget_bytes=budget, max_slots=8, device="cpu", tick_s=1e-3)
    assert out["requests"] == 3 and out["rejected"] == 0
    assert small.admitted < big.admitted
    assert big.admitted >= first.finished  # it waited for the memory of the first


def test_request_larger_than_the_budget_is_rejected(fakes):
    reqs = serve.poisson_requests(4, rate=1e4, seed=2, two_d=(64, 96), three_d=(16, 24), frac_2d=1.0)
    huge = serve.Request(99, reqs[-1].arrival, 2, 1024, 12.0, (0.5, 0.5), 9)
    budget = max(serve.workspace_bytes(r, cmcg.MIXED) for r in reqs) * 2
    assert serve.workspace_bytes(huge, cmcg.MIXED) > budget
    out = serve.serve(reqs + [huge], budget_bytes=budget, max_slots=4, device="cpu")
    assert out["requests"] == 4 and out["rejected"] == 1 and huge.rejected


def test_nothing_admissible_returns(fakes):
    reqs = serve.poisson_requests(2, rate=1e4, seed=4, two_d=(64, 96), three_d=(16, 24), frac_2d=1.0)
    out = serve.serve(reqs, budget_bytes=1, max_slots=4, device="cpu")
    assert out["requests"] == 0 and out["rejected"] == 2 and out["latency_ms"] is None
