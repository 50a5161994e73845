"""Oracle wave solver (test infrastructure only; see oracle/__init__.py).

Semi-discrete wave equation of Eq. WE after mass lumping:  M y'' + B y' + K y = F(t), with
initial data y(0) = v0, y'(0) = v1 (Eq. WE_INIT).  Time stepping: leapfrog (LF, Sec. 4.3.1)
with the absorbing term centred in time, run here in its velocity-Verlet (kick-drift-kick)
form, one step Phi: (y^n, v^n) -> (y^{n+1}, v^{n+1}):

    v^{n+1/2} = v^n + (dt/2) M^-1 (F^n - K y^n - B v^n)
    y^{n+1}   = y^n + dt v^{n+1/2}
    (M + (dt/2) B) v^{n+1} = M v^{n+1/2} + (dt/2) (F^{n+1} - K y^{n+1})

which is algebraically the three-level scheme
    M (y^{n+1} - 2 y^n + y^{n-1})/dt^2 + B (y^{n+1} - y^{n-1})/(2 dt) + K y^n = F^n.
The period map is Pi(w) = Phi^N(w) = P w + b (P linear, b = Pi(0)).

The energy functional of Eq. cost_functional_J, discretised with the lumped operators:
    J(v0, v1) = 1/2 e0.K e0 + 1/2 e1.M e1,   e = Pi(v) - v.

The transposed period P^T is written as the literal reverse of the three-level scheme's
computational graph (start half-kick, N-1 leapfrog steps, end velocity), which is the
discrete counterpart of the backward wave equation (Eq. AWE) needed for J' (Eq.
J1_derivative_final).

Parity: pinned by the discrete energy identity with closed and absorbing boundaries
(E^{n+1/2} - E^{n-1/2} = dt v^n.(F^n - B v^n)), by the dot-product test <P x, y> = <x, P^T y>,
and, through the CMCG fixed point, by the direct solve of the time-discrete Helmholtz system.
"""
from __future__ import annotations

import numpy as np

from .grid import Discretization


def step(dz: Discretization, y, v, n: int, F_hat=None):
    """One velocity-Verlet leapfrog step from t_n to t_{n+1}.  Returns (y', v', v_half)."""
    return kick_drift_kick(dz, y, v, dz.forcing(F_hat, n), dz.forcing(F_hat, n + 1))


def kick_drift_kick(dz: Discretization, y, v, Fn, Fn1):
    """The step with the loads F^n, F^{n+1} given as arrays.  Returns (y', v', v_half)."""
    dt = dz.dt
    v_half = v + (dt / 2.0) * (Fn - dz.K(y) - dz.B * v) / dz.M
    y_new = (y + dt * v_half) * dz.act
    v_new = (dz.M * v_half + (dt / 2.0) * (Fn1 - dz.K(y_new))) / (dz.M + (dt / 2.0) * dz.B)
    return y_new, v_new * dz.act, v_half * dz.act


def period(dz: Discretization, y0, v0, F_hat=None):
    """Pi(y0, v0): N steps over one period T.  F_hat is the complex load amplitude (or None)."""
    y = np.asarray(y0, dtype=np.float64).reshape(dz.shape) * dz.act
    v = np.asarray(v0, dtype=np.float64).reshape(dz.shape) * dz.act
    for n in range(dz.N):
        y, v, _ = step(dz, y, v, n, F_hat)
    return y, v


def theta_tr(t: float, t_tr: float) -> float:
    """Smooth switch-on of the sources for the initial run-up (Sec. 4.2.3, Eq. transientfunction):
    with s = sin(pi t / (2 t_tr)), theta = (2 - s) s on [0, t_tr] and 1 afterwards.  It rises
    from 0 at t = 0 to 1 at t = t_tr, where its slope vanishes."""
    if t >= t_tr:
        return 1.0
    s = np.sin(0.5 * np.pi * t / t_tr)
    return float((2.0 - s) * s)


def long_time(dz: Discretization, F_hat, periods: int, smooth: bool = True, trajectory: bool = False):
    """The forced wave equation (Eq. WE) integrated from rest, y(0) = y'(0) = 0, up to
    t = periods * T: the time-dependent solution w(., t) whose state at t = l T the
    do-nothing solver of Sec. 4.2 reads (Eq. AP_SOLUTION) and the initial run-up of Sec. 4.2.3
    hands to CMCG.  With smooth=True the load is theta_tr(t) F(t), t_tr = periods * T.
    Returns (y, v) at t = periods * T, and with trajectory=True also the list of every y^n."""
    total = periods * dz.N
    t_tr = total * dz.dt
    y = np.zeros(dz.shape)
    v = np.zeros(dz.shape)
    ys = [y]
    for n in range(total):
        th0 = theta_tr(n * dz.dt, t_tr) if smooth else 1.0
        th1 = theta_tr((n + 1) * dz.dt, t_tr) if smooth else 1.0
        y, v, _ = kick_drift_kick(dz, y, v, th0 * dz.forcing(F_hat, n), th1 * dz.forcing(F_hat, n + 1))
        if trajectory:
            ys.append(y)
    return (y, v, ys) if trajectory else (y, v)


def transposed_period(dz: Discretization, a, b):
    """P^T (a, b): the transpose of the homogeneous period map, written as the reverse of the
    three-level scheme's graph.  Notation: C = M - (dt/2)B, D = M + (dt/2)B.

      end      : v^N = D^-1 [M (y^N - y^{N-1})/dt - (dt/2) K y^N]
      steps    : y^{n+1} = D^-1 [(2M - dt^2 K) y^n - C y^{n-1}],   n = 1..N-1
      start    : y^1 = y^0 + dt v^0 - (dt^2/2) M^-1 (K y^0 + B v^0)
    Each line is transposed in reverse order, accumulating cotangents ybar_n."""
    dt, N = dz.dt, dz.N
    M, B = dz.M, dz.B
    C = M - (dt / 2.0) * B
    D = M + (dt / 2.0) * B
    a = np.asarray(a, dtype=np.float64).reshape(dz.shape) * dz.act
    b = np.asarray(b, dtype=np.float64).reshape(dz.shape) * dz.act
    ybar = [np.zeros(dz.shape) for _ in range(N + 1)]

    # end velocity
    t = b / D
    ybar[N] += a + M * t / dt - (dt / 2.0) * dz.K(t)
    ybar[N - 1] += -M * t / dt
    # leapfrog steps in reverse
    for n in range(N - 1, 0, -1):
        u = ybar[n + 1] / D
        ybar[n] += 2.0 * M * u - dt * dt * dz.K(u)
        ybar[n - 1] += -C * u
    # start half-kick
    y0bar = ybar[0] + ybar[1]
    vbar_h = dt * ybar[1]
    v0bar = vbar_h - (dt / 2.0) * B * vbar_h / M
    y0bar = y0bar - (dt / 2.0) * dz.K(vbar_h / M)
    return y0bar * dz.act, v0bar * dz.act


def energy_operator(dz: Discretization, e0, e1):
    """E e = (K e0, M e1): the discrete energy inner product of Eq. cost_functional_J."""
    return dz.K(e0), dz.M * e1 * dz.act


def energy(dz: Discretization, e0, e1) -> float:
    """J-type energy 1/2 e0.K e0 + 1/2 e1.M e1."""
    z0, z1 = energy_operator(dz, e0, e1)
    return 0.5 * float(np.sum(e0 * z0) + np.sum(e1 * z1))


def functional_J(dz: Discretization, v0, v1, F_hat=None) -> float:
    """J(v0, v1) of Eq. cost_functional_J: energy of the mismatch after one period."""
    yT, vT = period(dz, v0, v1, F_hat)
    return energy(dz, yT - v0 * dz.act, vT - v1 * dz.act)
