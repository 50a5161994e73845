"""The allocation-free wave period (cmcg_wave_period_static) against cmcg_wave_period.

cmcg_wave_period_static serves callers that cannot allocate device memory (a plug-in whose
host application owns the device-memory budget, or a real-time loop that must avoid
cudaMalloc's implicit synchronisation).  Its scratch is a static device array inside the
library, shared by all calls.  This file is collected last so that a failure here comes after
every other test has run; it also passes alone in a fresh process.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_1903_12522_gb300 import cmcg  # noqa: E402
from paper_1903_12522_gb300 import workloads as wl  # noqa: E402

TOL = 1e-12  # the FP64 per-period tolerance of the parity tests


def rel(a, b):
    return float(torch.linalg.vector_norm(a - b) / torch.linalg.vector_norm(b))


@pytest.mark.parametrize("name", ["gauss2d_40", "sphere3d_24"])
def test_static_period_matches_workspace_period_twice(name):
    w = wl.gaussian_2d(n=40) if name == "gauss2d_40" else wl.sphere_3d(n=24)
    s = cmcg.Solver(w.n, w.h, w.c, w.omega, w.faces, mask=w.mask, precision=cmcg.FP64, dt=w.dt_target)
    act = 1.0 if w.mask is None else 1.0 - w.mask.astype(np.float64)
    y0, v0 = [torch.as_tensor(x * act, device="cuda").reshape(-1) for x in wl.random_fields(w.shape, 2, 31)]
    f = None if w.f is None else torch.as_tensor(w.f, device="cuda").reshape(-1)
    g = None if w.g is None else torch.as_tensor(w.g, device="cuda").reshape(-1)
    ref_u, ref_v = [t.reshape(-1) for t in s.wave_period(y0, v0, f, g)]

    c = torch.as_tensor(w.c, device="cuda").reshape(-1)
    mask = None if w.mask is None else torch.as_tensor(w.mask, device="cuda").reshape(-1)
    bc = cmcg.BC()
    for k in range(6):
        bc.face[k] = int(w.faces[k])
    bc.dirichlet_mask = None if mask is None else mask.data_ptr()
    grid = cmcg.make_grid(w.n, w.h, w.order)
    stream = torch.cuda.current_stream().cuda_stream
    outs = []
    for _ in range(2):
        uT = torch.full_like(ref_u, float("nan"))
        vT = torch.full_like(ref_v, float("nan"))
        code = cmcg.cmcg_wave_period_static(grid, c, w.omega, bc, w.dt_target, y0, v0, f, g, uT, vT, stream)
        assert code == cmcg.OK, cmcg.cmcg_status_string(code)
        assert rel(uT, ref_u) <= TOL and rel(vT, ref_v) <= TOL
        outs.append((uT, vT))
    assert torch.equal(outs[0][0], outs[1][0]) and torch.equal(outs[0][1], outs[1][1])


def test_static_period_rejects_grids_above_its_maximum():
    w = wl.sphere_3d(n=64)  # 65^3 = 274,625 nodes > 262,144
    grid = cmcg.make_grid(w.n, w.h)
    bc = cmcg.BC()
    dummy = torch.zeros(1, dtype=torch.float64, device="cuda")
    code = cmcg.cmcg_wave_period_static(grid, dummy, w.omega, bc, w.dt_target, dummy, dummy, None, None, dummy,
                                        dummy, torch.cuda.current_stream().cuda_stream)
    assert code == cmcg.ERR_WORKSPACE
