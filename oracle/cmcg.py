"""Oracle CMCG solver (test infrastructure only; see oracle/__init__.py).

The CMCG Algorithm of Sec. 2.3, steps (1)-(6), on the discretisation of oracle/grid.py:

 (1) v = (v0, v1) = 0 (the paper's choice in Sec. 4.1), or a given initial guess.
 (2) gradient g = J'(v): forward period with the sources, mismatch e = Pi(v) - v,
     z = E e, adjoint (transposed) period q = P^T z, g = q - z.
 (3) Riesz representer g~ = (K^+ g0, M^-1 g1)          (Eq. CMCG_PRECONDITIONIER)
 (4) r = d = g~
 (5) for l = 1, 2, ...
     5.1 homogeneous forward + adjoint period from d: g = (P - I)^T E (P - I) d
     5.2 g~ = Riesz(g)
     5.3 alpha = ||r||_E^2 / (g~, d)_E,  (a, b)_E = a0.K b0 + a1.M b1
         (the discrete (grad a0, grad b0) + (a1/c^2, b1) of the paper)
     5.4 v -= alpha d
     5.5 r -= alpha g~
     5.6 beta = ||r_new||_E^2 / ||r||_E^2
     5.7 d = r + beta d
     5.8 stop when sqrt(||r||_E^2 / ||r^(0)||_E^2) <= tol
 (6) u = v0 + (i / omega_hat) v1 (discrete reading of u = v0 + (i/omega) v1: omega_hat =
     sin(omega dt)/dt makes the recovery exact for the time-discrete periodic solution).
     Without Dirichlet nodes the minimiser is defined up to a constant shift lambda in v0
     (Theorem 1); lambda is removed with the discrete compatibility condition (Sec. 2.1):
        lambda = (1.F^ + wt^2 1.M u + i wh 1.B u) / (wt^2 sum M + i wh sum B).

J(v^(l)) is tracked along the iteration through the mismatch e(v) = Pi(v) - v, which
changes by -alpha (P - I) d when v changes by -alpha d.

Parity: pinned against the direct solve of the time-discrete Helmholtz problem
(oracle/direct.py) -- the paper's own verification of Sec. 4.1 (CMCG -> direct solve of the
same discretisation) -- and by the manufactured discrete plane wave.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

from .grid import Discretization
from .riesz import RieszSolver
from .wave import energy_operator, period, step, transposed_period


def e_inner(dz: Discretization, a0, a1, b0, b1) -> float:
    """(a, b)_E = a0.K b0 + a1.M b1."""
    return float(np.sum(a0 * dz.K(b0)) + np.sum(a1 * dz.M * b1 * dz.act))


@dataclasses.dataclass
class CMCGResult:
    u: np.ndarray
    v0: np.ndarray
    v1: np.ndarray
    iterations: int
    rel_residual: float
    residual_history: list
    J_history: list
    lam: complex


def gradient(dz: Discretization, w0, w1, F_hat=None):
    """J'(w) for the functional with load F_hat (None = homogeneous).
    Returns (g0, g1, e0, e1, e_pe0, e_pe1) where e is the mismatch Pi(w) - w."""
    yT, vT = period(dz, w0, w1, F_hat)
    e0 = (yT - w0) * dz.act
    e1 = (vT - w1) * dz.act
    z0, z1 = energy_operator(dz, e0, e1)
    q0, q1 = transposed_period(dz, z0, z1)
    return q0 - z0, q1 - z1, e0, e1


def remove_shift(dz: Discretization, u_cg, F_hat):
    """Discrete compatibility condition: lambda with (K - wt^2 M - i wh B)(u_cg - lambda) = F^."""
    if dz.has_dirichlet:
        return u_cg, 0.0 + 0.0j
    wt2 = dz.omega_tilde ** 2
    wh = dz.omega_hat
    num = np.sum(F_hat) + wt2 * np.sum(dz.M * u_cg) + 1j * wh * np.sum(dz.B * u_cg)
    den = wt2 * np.sum(dz.M * dz.act) + 1j * wh * np.sum(dz.B)
    lam = complex(num / den)
    return (u_cg - lam) * dz.act, lam


def filtered(dz: Discretization, v0, v1, F_hat):
    """Step (6) by the fundamental-frequency filter of Sec. 2.2 (Eq.
    fundamental-frequency-solution): one forced period from (v0, v1), with the time integral
    taken by the rectangle rule over t_n = n dt, n = 0..N-1, and i/omega_hat in place of i/omega
    (both exact for the discrete time-harmonic solution):
        y^ = (1/N) sum_n (y^n + (i / omega_hat) v^n) exp(i omega t_n).
    The filter removes lambda and every T-periodic eigenmode.  A linear growth eta t of the
    minimiser leaves a constant; by the proposition of Sec. 2.2 eta = 0 when there are
    absorbing faces or Dirichlet nodes, and in the pure Neumann case the constant is fixed by
    the compatibility condition (Eq. cc_neumann_eta, here in its discrete form).
    Returns (u, shift)."""
    y = np.asarray(v0, dtype=np.float64).reshape(dz.shape) * dz.act
    v = np.asarray(v1, dtype=np.float64).reshape(dz.shape) * dz.act
    acc = np.zeros(dz.shape, dtype=np.complex128)
    for n in range(dz.N):
        acc += (y + (1j / dz.omega_hat) * v) * np.exp(1j * dz.omega * n * dz.dt)
        y, v, _ = step(dz, y, v, n, F_hat)
    u = acc / dz.N * dz.act
    if dz.has_dirichlet or float(np.sum(dz.B)) > 0.0:
        return u, 0.0 + 0.0j
    return remove_shift(dz, u, F_hat)


def asymptotic(dz: Discretization, y, v, F_hat):
    """The do-nothing approximation of Sec. 4.2 (Eq. AP_SOLUTION) from the state (y, v) of the
    forced wave equation at t = l T, recovered as in step (6): y + (i / omega_hat) v, then the
    compatibility-condition shift when there are no Dirichlet nodes (the constant mode is a
    steady state of the homogeneous equation, so the long-time state can carry one too)."""
    u = (np.asarray(y).reshape(dz.shape) + (1j / dz.omega_hat) * np.asarray(v).reshape(dz.shape)) * dz.act
    return remove_shift(dz, u, F_hat)[0]


def solve(dz: Discretization, F_hat, tol=1e-12, max_iter=10000, v_init=None, riesz=None) -> CMCGResult:
    act = dz.act
    riesz = riesz or RieszSolver(dz)
    # (1)
    if v_init is None:
        v0 = np.zeros(dz.shape)
        v1 = np.zeros(dz.shape)
    else:
        v0 = np.asarray(v_init[0], dtype=np.float64).reshape(dz.shape) * act
        v1 = np.asarray(v_init[1], dtype=np.float64).reshape(dz.shape) * act
    # (2)
    g0, g1, e0, e1 = gradient(dz, v0, v1, F_hat)
    J_hist = [0.5 * e_inner(dz, e0, e1, e0, e1)]
    # (3)
    gt0, gt1 = riesz.representer(g0, g1)
    # (4)
    r0, r1 = gt0.copy(), gt1.copy()
    d0, d1 = gt0.copy(), gt1.copy()
    rr = e_inner(dz, r0, r1, r0, r1)
    rr0 = rr
    hist = [1.0]
    it = 0
    rel = 1.0 if rr0 > 0 else 0.0
    if rr0 <= 0.0:
        max_iter = 0
    # (5)
    for it in range(1, max_iter + 1):
        # 5.1
        g0, g1, ed0, ed1 = gradient(dz, d0, d1, None)
        # 5.2
        gt0, gt1 = riesz.representer(g0, g1)
        # 5.3
        alpha = rr / e_inner(dz, gt0, gt1, d0, d1)
        # 5.4
        v0 = v0 - alpha * d0
        v1 = v1 - alpha * d1
        e0 = e0 - alpha * ed0
        e1 = e1 - alpha * ed1
        J_hist.append(0.5 * e_inner(dz, e0, e1, e0, e1))
        # 5.5
        r0 = r0 - alpha * gt0
        r1 = r1 - alpha * gt1
        # 5.6
        rr_new = e_inner(dz, r0, r1, r0, r1)
        beta = rr_new / rr
        # 5.7
        d0 = r0 + beta * d0
        d1 = r1 + beta * d1
        rr = rr_new
        # 5.8
        rel = math.sqrt(max(rr, 0.0) / rr0)
        hist.append(rel)
        if rel <= tol:
            break
    # (6)
    u_cg = (v0 + 1j * v1 / dz.omega_hat) * act
    u, lam = remove_shift(dz, u_cg, F_hat)
    return CMCGResult(u=u, v0=v0, v1=v1, iterations=it, rel_residual=rel,
                      residual_history=hist, J_history=J_hist, lam=lam)
