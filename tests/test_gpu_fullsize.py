"""Full-size checks of the 4th-order (13-point) path on the 513^3 layered-medium workload, by
properties that hold at any size (the oracle parity of the same kernels runs at small sizes in
test_gpu_parity.py): the FP32 period agrees with the FP64 period to FP32 accuracy, and the
FP64 adjoint passes the dot-product test."""
import math

import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_1903_12522_gb300 import cmcg  # noqa: E402
from paper_1903_12522_gb300 import workloads as wl  # noqa: E402


@pytest.fixture(scope="module")
def layered():
    w = wl.layered_3d(n=512)
    gen = torch.Generator(device="cuda")
    gen.manual_seed(41)
    fields = [torch.randn(w.num_nodes, generator=gen, device="cuda", dtype=torch.float64) for _ in range(4)]
    return w, fields


def rel(a, b):
    return float(torch.linalg.vector_norm(a - b) / torch.linalg.vector_norm(b))


def test_layered_513_fp32_period_matches_fp64(layered):
    w, (y0, v0, _, _) = layered
    f = torch.as_tensor(w.f, device="cuda").reshape(-1)
    out = {}
    for prec in (cmcg.FP64, cmcg.FP32):
        s = cmcg.Solver(w.n, w.h, w.c, w.omega, w.faces, order=4, precision=prec, dt=w.dt_target)
        assert s.info["steps_per_period"] == 57
        out[prec] = [t.reshape(-1) for t in s.wave_period(y0, v0, f, None)]
        s.close()
        del s
        torch.cuda.empty_cache()
    assert rel(out[cmcg.FP32][0], out[cmcg.FP64][0]) <= 5e-5
    assert rel(out[cmcg.FP32][1], out[cmcg.FP64][1]) <= 5e-5


def test_layered_513_adjoint_dot_product(layered):
    w, (x0, x1, y0, y1) = layered
    s = cmcg.Solver(w.n, w.h, w.c, w.omega, w.faces, order=4, precision=cmcg.FP64, dt=w.dt_target)
    p0, p1 = [t.reshape(-1) for t in s.wave_period(x0, x1)]
    q0, q1 = [t.reshape(-1) for t in s.adjoint_period(y0, y1)]
    lhs = float(torch.dot(p0, y0) + torch.dot(p1, y1))
    rhs = float(torch.dot(x0, q0) + torch.dot(x1, q1))
    scale = math.sqrt(float(torch.dot(p0, p0) + torch.dot(p1, p1))) * math.sqrt(float(torch.dot(y0, y0) + torch.dot(y1, y1)))
    assert abs(lhs - rhs) <= 1e-12 * scale
    s.close()
