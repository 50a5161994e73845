"""Thin ctypes binding of libcmcg (C ABI in include/cmcg.h).

Argument marshalling only: every step of the solver runs in the CUDA library.  Torch is used
for device memory and streams.  The functions keep the C names (cmcg_create, cmcg_wave_period,
cmcg_solve, ...); ``Solver`` bundles a handle with its workspace.

Loading fails loudly (``RuntimeError``) when libcmcg.so has not been built; there is no CPU
fallback.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Optional

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libcmcg.so")
# the same library with the kernels' compiled-in bounds checks (build(checked=True)); loaded
# instead of LIB_PATH when the environment sets CMCG_CHECKED=1
LIB_CHECKED_PATH = os.path.join(HERE, "libcmcg_checked.so")

OK, NOT_CONVERGED = 0, 1
ERR_INVALID_ARG, ERR_CFL, ERR_WORKSPACE, ERR_UNSUPPORTED, ERR_CUDA, ERR_DIVERGED = -1, -2, -3, -4, -5, -6
BC_ABC, BC_NEUMANN, BC_DIRICHLET = 0, 1, 2
FP64, FP32, MIXED = 0, 1, 2
FLAG_HOST_IO = 1
FLAG_TIMING = 2
FLAG_INEXACT_RIESZ = 4
FLAG_FILTER = 8
FLAG_NO_CG = 16
FLAG_FIRST_ORDER = 32
FLAG_L2_KAPPA = 64

ERR_DEVICE_TIMEOUT = -7
ENGINE_NO_GRAPH = 1

EXPORTED = (
    "cmcg_workspace_size", "cmcg_create", "cmcg_destroy", "cmcg_get_info", "cmcg_get_history", "cmcg_wave_period",
    "cmcg_adjoint_period", "cmcg_riesz", "cmcg_solve", "cmcg_solve_warm", "cmcg_solve_host", "cmcg_status_string",
    "cmcg_engine_workspace_size", "cmcg_engine_create", "cmcg_engine_destroy", "cmcg_engine_submit",
    "cmcg_engine_tick", "cmcg_engine_result", "cmcg_engine_active", "cmcg_engine_info", "cmcg_engine_set_shape",
    "cmcg_engine_barrier_selftest", "cmcg_engine_cuda_error", "cmcg_fo_period", "cmcg_fo_adjoint_period",
    "cmcg_bulk_wait_selftest", "cmcg_check_status",
)


class Grid(C.Structure):
    _fields_ = [("dim", C.c_int), ("n", C.c_int * 3), ("h", C.c_double), ("order", C.c_int)]


class BC(C.Structure):
    _fields_ = [("face", C.c_ubyte * 6), ("dirichlet_mask", C.c_void_p)]


class Options(C.Structure):
    _fields_ = [("precision", C.c_int), ("dt", C.c_double), ("max_iter", C.c_int), ("riesz_tol", C.c_double),
                ("riesz_max_iter", C.c_int), ("inner_tol", C.c_double), ("flags", C.c_int),
                ("runup_periods", C.c_int), ("tile", C.c_int * 4)]


class Stats(C.Structure):
    _fields_ = [("iterations", C.c_int), ("outer_iterations", C.c_int), ("periods", C.c_int),
                ("riesz_iterations", C.c_int), ("steps_per_period", C.c_int), ("dt", C.c_double),
                ("omega_tilde", C.c_double), ("omega_hat", C.c_double), ("rel_residual", C.c_double),
                ("J0", C.c_double), ("J_final", C.c_double), ("lambda_re", C.c_double),
                ("lambda_im", C.c_double), ("point_updates", C.c_longlong), ("seconds", C.c_double),
                ("kernel_launches", C.c_longlong), ("runup_periods", C.c_int), ("step_seconds_fp32", C.c_double),
                ("step_seconds_fp64", C.c_double), ("step_launches_fp32", C.c_longlong),
                ("step_launches_fp64", C.c_longlong), ("graph_replays", C.c_longlong)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class Info(C.Structure):
    _fields_ = [("steps_per_period", C.c_int), ("dt", C.c_double), ("omega_tilde", C.c_double),
                ("omega_hat", C.c_double), ("num_nodes", C.c_longlong), ("mg_levels", C.c_int),
                ("has_dirichlet", C.c_int)]


_lib = None


def load(path: str = None):
    """Load libcmcg.so (libcmcg_checked.so when CMCG_CHECKED=1) and declare its signatures.
    Raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if path is None:
        path = LIB_CHECKED_PATH if os.environ.get("CMCG_CHECKED") == "1" else LIB_PATH
    if not os.path.exists(path):
        raise RuntimeError(f"{os.path.basename(path)} not built ({path}); run __graft_entry__.build()")
    lib = C.CDLL(path)
    P, I, D, S = C.c_void_p, C.c_int, C.c_double, C.c_size_t
    lib.cmcg_workspace_size.argtypes = [C.POINTER(Grid), C.POINTER(Options)]
    lib.cmcg_workspace_size.restype = S
    lib.cmcg_create.argtypes = [C.POINTER(Grid), P, D, C.POINTER(BC), C.POINTER(Options), P, S, P, C.POINTER(P)]
    lib.cmcg_create.restype = I
    lib.cmcg_destroy.argtypes = [P]
    lib.cmcg_destroy.restype = I
    lib.cmcg_get_info.argtypes = [P, C.POINTER(Info)]
    lib.cmcg_get_info.restype = I
    lib.cmcg_get_history.argtypes = [P, P, I, C.POINTER(I)]
    lib.cmcg_get_history.restype = I
    lib.cmcg_wave_period.argtypes = [P, P, P, P, P, P, P]
    lib.cmcg_wave_period.restype = I
    lib.cmcg_adjoint_period.argtypes = [P, P, P, P, P]
    lib.cmcg_adjoint_period.restype = I
    lib.cmcg_bulk_wait_selftest.argtypes = [I, P]
    lib.cmcg_bulk_wait_selftest.restype = I
    lib.cmcg_fo_period.argtypes = [P, P, P, P, P]
    lib.cmcg_fo_period.restype = I
    lib.cmcg_fo_adjoint_period.argtypes = [P, P, P]
    lib.cmcg_fo_adjoint_period.restype = I
    lib.cmcg_riesz.argtypes = [P, P, P]
    lib.cmcg_riesz.restype = I
    lib.cmcg_solve.argtypes = [P, P, P, D, P, C.POINTER(Stats)]
    lib.cmcg_solve.restype = I
    lib.cmcg_solve_warm.argtypes = [P, P, P, D, P, C.POINTER(Stats)]
    lib.cmcg_solve_warm.restype = I
    lib.cmcg_solve_host.argtypes = [P, P, P, D, P, C.POINTER(Stats)]
    lib.cmcg_solve_host.restype = I
    lib.cmcg_status_string.argtypes = [I]
    lib.cmcg_status_string.restype = C.c_char_p
    lib.cmcg_engine_workspace_size.argtypes = [I]
    lib.cmcg_engine_workspace_size.restype = S
    lib.cmcg_engine_create.argtypes = [I, P, S, P, I, C.POINTER(P)]
    lib.cmcg_engine_create.restype = I
    lib.cmcg_engine_destroy.argtypes = [P]
    lib.cmcg_engine_destroy.restype = I
    lib.cmcg_engine_set_shape.argtypes = [P, I, I]
    lib.cmcg_engine_set_shape.restype = I
    lib.cmcg_engine_submit.argtypes = [P, P, P, P, D, P]
    lib.cmcg_engine_submit.restype = I
    lib.cmcg_engine_tick.argtypes = [P, C.POINTER(I), I, C.POINTER(I)]
    lib.cmcg_engine_tick.restype = I
    lib.cmcg_engine_result.argtypes = [P, I, C.POINTER(Stats)]
    lib.cmcg_engine_result.restype = I
    lib.cmcg_engine_active.argtypes = [P]
    lib.cmcg_engine_active.restype = I
    lib.cmcg_engine_info.argtypes = [P, C.POINTER(C.c_longlong), C.POINTER(C.c_longlong)]
    lib.cmcg_engine_info.restype = I
    lib.cmcg_engine_barrier_selftest.argtypes = [P, C.c_longlong]
    lib.cmcg_engine_barrier_selftest.restype = I
    lib.cmcg_engine_cuda_error.argtypes = [P]
    lib.cmcg_engine_cuda_error.restype = C.c_char_p
    LL = C.POINTER(C.c_longlong)
    lib.cmcg_check_status.argtypes = [LL, LL, LL]
    lib.cmcg_check_status.restype = I
    _lib = lib
    return lib


class CMCGError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        msg = load().cmcg_status_string(code).decode()
        super().__init__(f"{where}: {msg} ({code})")


def _check(code: int, where: str, allow_not_converged: bool = False) -> int:
    if code == OK or (allow_not_converged and code == NOT_CONVERGED):
        return code
    raise CMCGError(code, where)


def _ptr(t) -> Optional[int]:
    return None if t is None else int(t.data_ptr())


def make_grid(n, h, order=2) -> Grid:
    g = Grid()
    g.dim = len(n)
    for a in range(3):
        g.n[a] = int(n[a]) if a < len(n) else 0
    g.h = float(h)
    g.order = int(order)
    return g


def make_options(precision=FP64, dt=0.0, max_iter=0, riesz_tol=0.0, riesz_max_iter=0, inner_tol=0.0, flags=0,
                 runup_periods=0, tile=None):
    o = Options()
    o.precision, o.dt, o.max_iter = int(precision), float(dt), int(max_iter)
    o.riesz_tol, o.riesz_max_iter, o.inner_tol, o.flags = float(riesz_tol), int(riesz_max_iter), float(inner_tol), int(flags)
    o.runup_periods = int(runup_periods)
    for k, v in enumerate(tile or ()):
        o.tile[k] = int(v)
    return o


# ---- C-named entry points -----------------------------------------------------------------
def cmcg_workspace_size(grid: Grid, opts: Options) -> int:
    return int(load().cmcg_workspace_size(C.byref(grid), C.byref(opts)))


def cmcg_create(grid: Grid, c, omega: float, bc: BC, opts: Options, workspace, stream) -> C.c_void_p:
    h = C.c_void_p()
    code = load().cmcg_create(C.byref(grid), _ptr(c), float(omega), C.byref(bc), C.byref(opts), _ptr(workspace),
                              int(workspace.numel() * workspace.element_size()), stream, C.byref(h))
    _check(code, "cmcg_create")
    return h


def cmcg_destroy(h) -> None:
    _check(load().cmcg_destroy(h), "cmcg_destroy")


def cmcg_get_info(h) -> dict:
    info = Info()
    _check(load().cmcg_get_info(h, C.byref(info)), "cmcg_get_info")
    return {k: getattr(info, k) for k, _ in info._fields_}


def cmcg_get_history(h) -> np.ndarray:
    """Relative residual per CG iteration of the handle's last solve (see include/cmcg.h)."""
    n = C.c_int(0)
    _check(load().cmcg_get_history(h, None, 0, C.byref(n)), "cmcg_get_history")
    out = np.zeros(n.value, dtype=np.float64)
    if n.value:
        _check(load().cmcg_get_history(h, out.ctypes.data, n.value, C.byref(n)), "cmcg_get_history")
    return out


def cmcg_wave_period(h, u0, v0, f, g, uT, vT) -> None:
    _check(load().cmcg_wave_period(h, _ptr(u0), _ptr(v0), _ptr(f), _ptr(g), _ptr(uT), _ptr(vT)), "cmcg_wave_period")


def cmcg_adjoint_period(h, a, b, q0, q1) -> None:
    _check(load().cmcg_adjoint_period(h, _ptr(a), _ptr(b), _ptr(q0), _ptr(q1)), "cmcg_adjoint_period")


def cmcg_bulk_wait_selftest(spin_limit: int, stream=None) -> int:
    """Bounded-wait self-test of the bulk-copy step kernel; returns the status code
    (ERR_DEVICE_TIMEOUT is the expected outcome)."""
    return int(load().cmcg_bulk_wait_selftest(int(spin_limit), stream))


def cmcg_check_status():
    """(code, count, site, index) of the compiled-in bounds checks since the last call; code is
    OK in the checked library and ERR_UNSUPPORTED in the normal one."""
    c, si, ix = C.c_longlong(), C.c_longlong(), C.c_longlong()
    code = load().cmcg_check_status(C.byref(c), C.byref(si), C.byref(ix))
    return int(code), int(c.value), int(si.value), int(ix.value)


def cmcg_fo_period(h, s0, f, g, sT) -> None:
    _check(load().cmcg_fo_period(h, _ptr(s0), _ptr(f), _ptr(g), _ptr(sT)), "cmcg_fo_period")


def cmcg_fo_adjoint_period(h, y, out) -> None:
    _check(load().cmcg_fo_adjoint_period(h, _ptr(y), _ptr(out)), "cmcg_fo_adjoint_period")


def cmcg_riesz(h, rhs, s) -> int:
    return _check(load().cmcg_riesz(h, _ptr(rhs), _ptr(s)), "cmcg_riesz", allow_not_converged=True)


def cmcg_solve(h, f, g, tol, u, stats: Optional[Stats] = None) -> int:
    st = stats if stats is not None else Stats()
    return _check(load().cmcg_solve(h, _ptr(f), _ptr(g), float(tol), _ptr(u), C.byref(st)), "cmcg_solve",
                  allow_not_converged=True)


def cmcg_solve_warm(h, f, g, tol, u, stats: Optional[Stats] = None) -> int:
    """cmcg_solve started from the field in u (complex, device); u receives the solution."""
    st = stats if stats is not None else Stats()
    return _check(load().cmcg_solve_warm(h, _ptr(f), _ptr(g), float(tol), _ptr(u), C.byref(st)), "cmcg_solve_warm",
                  allow_not_converged=True)


def cmcg_solve_host(h, f_host: Optional[np.ndarray], g_host: Optional[np.ndarray], tol, u_host: np.ndarray,
                    stats: Optional[Stats] = None) -> int:
    def hp(a):
        if a is None:
            return None
        assert a.dtype == np.complex128 and a.flags.c_contiguous
        return a.ctypes.data
    st = stats if stats is not None else Stats()
    return _check(load().cmcg_solve_host(h, hp(f_host), hp(g_host), float(tol), hp(u_host), C.byref(st)),
                  "cmcg_solve_host", allow_not_converged=True)


def cmcg_status_string(code: int) -> str:
    return load().cmcg_status_string(int(code)).decode()


def cmcg_wave_period_static(grid: Grid, c, omega, bc: BC, dt, u0, v0, f, g, uT, vT, stream) -> int:
    """The allocation-free FP64 period (static scratch inside the library); returns the status."""
    lib = load()
    fn = lib.cmcg_wave_period_static
    P = C.c_void_p
    fn.argtypes = [C.POINTER(Grid), P, C.c_double, C.POINTER(BC), C.c_double, P, P, P, P, P, P, P]
    fn.restype = C.c_int
    return int(fn(C.byref(grid), _ptr(c), float(omega), C.byref(bc), float(dt), _ptr(u0), _ptr(v0), _ptr(f),
                  _ptr(g), _ptr(uT), _ptr(vT), stream))


# ---- convenience wrapper ------------------------------------------------------------------
class Solver:
    """A handle plus its caller-owned workspace (torch uint8 tensor on the device)."""

    def __init__(self, n, h, c, omega, faces, mask=None, order=2, precision=FP64, dt=0.0, max_iter=0,
                 riesz_tol=0.0, riesz_max_iter=0, inner_tol=0.0, flags=0, device="cuda", stream=None,
                 runup_periods=0, tile=None):
        import torch

        load()
        self.torch = torch
        self.device = torch.device(device)
        self.n = tuple(int(m) for m in n)
        self.shape = tuple(m + 1 for m in reversed(self.n))
        self.grid = make_grid(self.n, h, order)
        if tile is None:
            from . import autotune

            tile = autotune.lookup(len(self.n), max(self.n), precision)
        self.opts = make_options(precision, dt, max_iter, riesz_tol, riesz_max_iter, inner_tol, flags, runup_periods,
                                 tile)
        nbytes = cmcg_workspace_size(self.grid, self.opts)
        if nbytes == 0:
            raise CMCGError(ERR_INVALID_ARG, "cmcg_workspace_size")
        self.workspace = torch.empty(nbytes, dtype=torch.uint8, device=self.device)
        self.c = self._dev(c, torch.float64)
        self.bc = BC()
        for f in range(6):
            self.bc.face[f] = int(faces[f])
        self.mask = None if mask is None else self._dev(mask, torch.uint8)
        self.bc.dirichlet_mask = _ptr(self.mask)
        # a stream of its own by default: the CG loop replays a captured CUDA graph, which the
        # legacy default stream does not allow
        self.stream = stream if stream is not None else torch.cuda.Stream(self.device)
        for t in (self.workspace, self.c, self.mask):
            if t is not None:
                t.record_stream(self.stream)
        self._after_caller()
        self.handle = cmcg_create(self.grid, self.c, omega, self.bc, self.opts, self.workspace, self.stream.cuda_stream)
        self.info = cmcg_get_info(self.handle)

    def _after_caller(self):
        # inputs produced on the caller's stream must be complete before this solver's stream
        # reads them (torch's side streams do not synchronise with the default stream)
        cur = self.torch.cuda.current_stream(self.device)
        if cur.cuda_stream != self.stream.cuda_stream:
            self.stream.wait_stream(cur)

    def _before_caller(self):
        cur = self.torch.cuda.current_stream(self.device)
        if cur.cuda_stream != self.stream.cuda_stream:
            cur.wait_stream(self.stream)

    def _dev(self, a, dtype):
        torch = self.torch
        if a is None:
            return None
        if isinstance(a, torch.Tensor):
            return a.to(device=self.device, dtype=dtype).contiguous().reshape(-1)
        # writeable C-contiguous host array (torch does not take read-only numpy buffers)
        return torch.as_tensor(np.require(a, requirements=["C", "W"])).to(device=self.device, dtype=dtype).reshape(-1)

    def close(self):
        if getattr(self, "handle", None) is not None:
            self.stream.synchronize()
            cmcg_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def wave_period(self, u0, v0, f=None, g=None):
        torch = self.torch
        u0, v0 = self._dev(u0, torch.float64), self._dev(v0, torch.float64)
        f, g = self._dev(f, torch.complex128), self._dev(g, torch.complex128)
        uT, vT = torch.empty_like(u0), torch.empty_like(v0)
        self._after_caller()
        cmcg_wave_period(self.handle, u0, v0, f, g, uT, vT)
        self._before_caller()
        return uT.reshape(self.shape), vT.reshape(self.shape)

    def adjoint_period(self, a, b):
        torch = self.torch
        a, b = self._dev(a, torch.float64), self._dev(b, torch.float64)
        q0, q1 = torch.empty_like(a), torch.empty_like(b)
        self._after_caller()
        cmcg_adjoint_period(self.handle, a, b, q0, q1)
        self._before_caller()
        return q0.reshape(self.shape), q1.reshape(self.shape)

    def fo_period(self, s0, f=None, g=None):
        """First-order handles: one forward period of the state (p_x, p_y[, p_z], v), flattened
        to (dim + 1) * N_p doubles."""
        torch = self.torch
        s0 = self._dev(s0, torch.float64)
        f, g = self._dev(f, torch.complex128), self._dev(g, torch.complex128)
        sT = torch.empty_like(s0)
        self._after_caller()
        cmcg_fo_period(self.handle, s0, f, g, sT)
        self._before_caller()
        return sT

    def fo_adjoint_period(self, y):
        torch = self.torch
        y = self._dev(y, torch.float64)
        out = torch.empty_like(y)
        self._after_caller()
        cmcg_fo_adjoint_period(self.handle, y, out)
        self._before_caller()
        return out

    def riesz(self, rhs):
        torch = self.torch
        rhs = self._dev(rhs, torch.float64)
        s = torch.empty_like(rhs)
        self._after_caller()
        code = cmcg_riesz(self.handle, rhs, s)
        self._before_caller()
        return s.reshape(self.shape), code

    def history(self):
        """Relative residual per CG iteration of the last solve."""
        return cmcg_get_history(self.handle)

    def solve(self, f=None, g=None, tol=1e-6, u0=None):
        """Solve; u0 (optional) is a start field (a checkpointed iterate, a nearby solution)."""
        torch = self.torch
        f, g = self._dev(f, torch.complex128), self._dev(g, torch.complex128)
        if u0 is None:
            u = torch.empty(int(np.prod(self.shape)), dtype=torch.complex128, device=self.device)
        else:
            u = self._dev(u0, torch.complex128).clone()
        st = Stats()
        self._after_caller()
        code = (cmcg_solve(self.handle, f, g, tol, u, st) if u0 is None
                else cmcg_solve_warm(self.handle, f, g, tol, u, st))
        self._before_caller()
        out = st.as_dict()
        out["status"] = code
        return u.reshape(self.shape), out


# ---- multi-solve engine ----------------------------------------------------------------------
class Engine:
    """Batched / served solves: a cmcg_engine plus its device workspace.  Solvers submitted to it
    must share its stream and use precision FP32 or MIXED with FLAG_INEXACT_RIESZ.  Without a
    stream argument the engine creates its own (CUDA graphs need a created stream); pass
    engine.stream to the solvers."""

    def __init__(self, max_slots, stream=None, flags=0, device="cuda", shape=None):
        import torch

        lib = load()
        self.torch = torch
        self.device = torch.device(device)
        self.stream = stream if stream is not None else torch.cuda.Stream(self.device)
        nbytes = int(lib.cmcg_engine_workspace_size(int(max_slots)))
        if nbytes == 0:
            raise CMCGError(ERR_INVALID_ARG, "cmcg_engine_workspace_size")
        self.workspace = torch.empty(nbytes, dtype=torch.uint8, device=self.device)
        self.handle = C.c_void_p()
        _check(lib.cmcg_engine_create(int(max_slots), self.workspace.data_ptr(), nbytes, self.stream.cuda_stream,
                                      int(flags), C.byref(self.handle)), "cmcg_engine_create")
        self.max_slots = int(max_slots)
        self._pending = {}
        if shape is not None:
            self.set_shape(*shape)

    def set_shape(self, blocks_per_sm=0, z_planes=0):
        """Launch shape of the batched step kernel (cmcg_engine_set_shape); only while idle."""
        _check(load().cmcg_engine_set_shape(self.handle, int(blocks_per_sm), int(z_planes)),
               "cmcg_engine_set_shape")

    def close(self):
        if getattr(self, "handle", None) is not None and self.handle.value:
            load().cmcg_engine_destroy(self.handle)
            self.handle = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def submit(self, solver, f=None, g=None, tol=1e-6):
        """Admit a solve; returns its slot.  The result tensor is returned by result()."""
        torch = self.torch
        f, g = solver._dev(f, torch.complex128), solver._dev(g, torch.complex128)
        u = torch.empty(int(np.prod(solver.shape)), dtype=torch.complex128, device=self.device)
        cur = torch.cuda.current_stream(self.device)
        if cur.cuda_stream != self.stream.cuda_stream:
            self.stream.wait_stream(cur)
        slot = load().cmcg_engine_submit(self.handle, solver.handle, _ptr(f), _ptr(g), float(tol), _ptr(u))
        if slot < 0:
            raise CMCGError(slot, "cmcg_engine_submit")
        self._pending[slot] = (solver, u, f, g)
        return slot

    def tick(self):
        """One CG iteration of every active solve; returns the slots that finished."""
        buf = (C.c_int * self.max_slots)()
        n = C.c_int(0)
        code = load().cmcg_engine_tick(self.handle, buf, self.max_slots, C.byref(n))
        if code != OK:
            raise CMCGError(code, "cmcg_engine_tick [" + load().cmcg_engine_cuda_error(self.handle).decode() + "]")
        return [buf[i] for i in range(n.value)]

    def result(self, slot):
        st = Stats()
        code = load().cmcg_engine_result(self.handle, int(slot), C.byref(st))
        solver, u, _, _ = self._pending.pop(slot)
        cur = self.torch.cuda.current_stream(self.device)
        if cur.cuda_stream != self.stream.cuda_stream:
            cur.wait_stream(self.stream)
        out = st.as_dict()
        out["status"] = code
        return u.reshape(solver.shape), out

    def active(self):
        return int(load().cmcg_engine_active(self.handle))

    def info(self):
        t, gb = C.c_longlong(0), C.c_longlong(0)
        load().cmcg_engine_info(self.handle, C.byref(t), C.byref(gb))
        return {"ticks": t.value, "graph_builds": gb.value}

    def barrier_selftest(self, spin_limit=100000):
        return int(load().cmcg_engine_barrier_selftest(self.handle, int(spin_limit)))

    def run_all(self):
        """Tick until every admitted solve has finished; returns {slot: (u, stats)}."""
        out = {}
        while self.active() > 0:
            for s in self.tick():
                out[s] = self.result(s)
        return out
