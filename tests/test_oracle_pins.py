"""Pins of the CPU oracle to facts fixed by the paper and by the mathematics, not by itself.

Each test names the fact it checks.  None of these tests needs a GPU.
"""
import math

import numpy as np
import pytest

from oracle import cmcg, direct, first_order, wave
from oracle.grid import ABC, DIRICHLET, NEUMANN, Discretization
from paper_1903_12522_gb300 import workloads as wl


def make(w: wl.Workload) -> Discretization:
    return Discretization(w.n, w.h, w.c, w.omega, w.faces, w.dt_target, order=w.order, mask=w.mask)


def wnorm(dz, a):
    return math.sqrt(float(np.sum(dz.W * dz.act * np.abs(a) ** 2)))


def rel_err(dz, a, b):
    return wnorm(dz, a - b) / wnorm(dz, b)


def cosine_mode(n, h, ks):
    xs = wl.coords(n, h)
    out = 1.0
    for a, k in enumerate(ks):
        out = out * np.cos(math.pi * k * xs[a] / (n[a] * h))
    return out * np.ones(tuple(m + 1 for m in reversed(n)))


def neumann_symbol(order, h, n_a, k):
    th = math.pi * k / n_a
    if order == 2:
        return 4.0 / h ** 2 * math.sin(th / 2.0) ** 2
    return (2.5 - (8.0 / 3.0) * math.cos(th) + (1.0 / 6.0) * math.cos(2 * th)) / h ** 2


def box(n, order=2, c=None, faces=None, omega=3.0, dt_frac=0.3, mask=None):
    h = 1.0 / max(n)
    shape = tuple(m + 1 for m in reversed(n))
    c = np.ones(shape) if c is None else c
    faces = faces or (ABC,) * 6
    return Discretization(n, h, c, omega, faces, dt_frac * h, order=order, mask=mask)


# ----------------------------------------------------------------------------------------
# P5a: the stiffness K is W times the Neumann (mirror) Laplacian; every cosine mode
# prod_a cos(pi k_a j_a / n_a) is an eigenvector with eigenvalue sum_a symbol(k_a).
# Closed form of the textbook Neumann problem; a wrong boundary weight, a transposed axis or
# a wrong 4th-order coefficient fails it.
@pytest.mark.parametrize("n,order", [((6, 9), 2), ((4, 5, 7), 2), ((8, 10), 4), ((6, 7, 5), 4)])
def test_K_cosine_eigenmodes(n, order):
    dz = box(n, order=order, faces=(NEUMANN,) * 6)
    rng = np.random.default_rng(1)
    for _ in range(12):
        ks = [int(rng.integers(0, m + 1)) for m in n]
        phi = cosine_mode(n, dz.h, ks)
        lam = sum(neumann_symbol(order, dz.h, n[a], ks[a]) for a in range(len(n)))
        lhs = dz.K(phi)
        rhs = dz.W * lam * phi
        scale = max(np.abs(rhs).max(), dz.W.max() / dz.h ** 2)
        assert np.abs(lhs - rhs).max() <= 1e-12 * scale, (ks, order)


# P5b: Riesz map on an obstacle-free box = closed-form cosine synthesis with W-mean zero.
@pytest.mark.parametrize("n", [(8, 12), (6, 4, 8)])
def test_riesz_closed_form(n):
    from oracle.riesz import RieszSolver

    dz = box(n)
    rng = np.random.default_rng(2)
    s_true = np.zeros(dz.shape)
    rhs = np.zeros(dz.shape)
    for _ in range(6):
        ks = [int(rng.integers(0, m + 1)) for m in n]
        if all(k == 0 for k in ks):
            continue
        a = rng.standard_normal()
        phi = cosine_mode(n, dz.h, ks)
        lam = sum(neumann_symbol(2, dz.h, n[ax], ks[ax]) for ax in range(len(n)))
        s_true += a * phi
        rhs += a * lam * dz.W * phi
    s = RieszSolver(dz).solve(rhs)
    assert abs(float(np.sum(dz.W * s))) <= 1e-13 * wnorm(dz, s_true)
    assert rel_err(dz, s, s_true) <= 1e-12


def test_riesz_dirichlet_residual():
    from oracle.riesz import RieszSolver

    w = wl.sphere_3d(n=8)
    dz = make(w)
    rhs = np.random.default_rng(3).standard_normal(dz.shape) * dz.act
    s = RieszSolver(dz).solve(rhs)
    assert np.all(s[dz.dirichlet] == 0)
    assert np.linalg.norm(dz.K(s) - rhs) <= 1e-12 * np.linalg.norm(rhs)


# ----------------------------------------------------------------------------------------
# P2: discrete energy identity of leapfrog.  With E^{n+1/2} = 1/2 v^{n+1/2}.M v^{n+1/2}
# + 1/2 y^n.K y^{n+1}: E^{n+1/2} - E^{n-1/2} = dt v^n.(F^n - B v^n), v^n = (v^{n-1/2}+v^{n+1/2})/2.
@pytest.mark.parametrize("closed", [True, False])
def test_energy_identity(closed):
    n = (10, 8, 6)
    shape = tuple(m + 1 for m in reversed(n))
    rng = np.random.default_rng(4)
    c = 1.0 + 0.3 * rng.random(shape)
    faces = (NEUMANN,) * 6 if closed else (ABC, ABC, NEUMANN, ABC, ABC, NEUMANN)
    dz = box(n, c=c, faces=faces, omega=5.0, dt_frac=0.25)
    F_hat = None if closed else dz.load(rng.standard_normal(shape) + 1j * rng.standard_normal(shape), None)
    y = rng.standard_normal(shape)
    v = rng.standard_normal(shape)
    E_prev = None
    vh_prev = None
    y_prev = None
    E0 = None
    for n_step in range(dz.N):
        y_new, v_new, vh = wave.step(dz, y, v, n_step, F_hat)
        E = 0.5 * np.sum(vh * dz.M * vh) + 0.5 * np.sum(y * dz.K(y_new))
        if E0 is None:
            E0 = abs(E)
        if E_prev is not None:
            vn = 0.5 * (vh_prev + vh)
            Fn = dz.forcing(F_hat, n_step)
            expected = dz.dt * np.sum(vn * (Fn - dz.B * vn))
            assert abs((E - E_prev) - expected) <= 1e-13 * E0
        E_prev, vh_prev, y_prev = E, vh, y
        y, v = y_new, v_new
    if closed:
        assert abs(E_prev - E0) <= 1e-13 * dz.N * E0


# ----------------------------------------------------------------------------------------
# P4: <P x, y> = <x, P^T y> for the homogeneous period map.
@pytest.mark.parametrize("case", ["abc2d", "mixed2d", "sphere3d", "order4"])
def test_adjoint_dot_product(case):
    if case == "abc2d":
        w = wl.gaussian_2d(n=12)
        dz = make(w)
    elif case == "mixed2d":
        n = (10, 13)
        c = 1.0 + 0.5 * np.random.default_rng(5).random((14, 11))
        dz = box(n, c=c, faces=(ABC, DIRICHLET, NEUMANN, ABC, ABC, ABC))
    elif case == "sphere3d":
        dz = make(wl.sphere_3d(n=8))
    else:
        dz = box((6, 7, 8), order=4, dt_frac=0.2)
    rng = np.random.default_rng(6)
    x0, x1, y0, y1 = [rng.standard_normal(dz.shape) * dz.act for _ in range(4)]
    p0, p1 = wave.period(dz, x0, x1)
    q0, q1 = wave.transposed_period(dz, y0, y1)
    lhs = np.sum(p0 * y0) + np.sum(p1 * y1)
    rhs = np.sum(x0 * q0) + np.sum(x1 * q1)
    scale = math.sqrt(np.sum(p0 ** 2) + np.sum(p1 ** 2)) * math.sqrt(np.sum(y0 ** 2) + np.sum(y1 ** 2))
    assert abs(lhs - rhs) <= 1e-13 * scale


# ----------------------------------------------------------------------------------------
# P1: CMCG converges to the direct solve of the same (time-)discretisation -- the paper's own
# verification (Sec. 4.1, tol 1e-14 there).
def _p1_cases():
    return ["gauss2d_8", "gauss2d_16", "sphere3d_8", "order4_3d", "mixed2d_hetero"]


@pytest.mark.parametrize("case", _p1_cases())
def test_cmcg_matches_direct(case):
    if case.startswith("gauss2d"):
        w = wl.gaussian_2d(n=int(case.split("_")[1]))
        dz, F = make(w), None
        F = dz.load(w.f, w.g)
    elif case == "sphere3d_8":
        w = wl.sphere_3d(n=8)
        dz = make(w)
        F = dz.load(w.f, w.g)
    elif case == "order4_3d":
        w = wl.layered_3d(n=8)
        dz = make(w)
        F = dz.load(w.f, w.g)
    else:
        n = (12, 10)
        rng = np.random.default_rng(7)
        c = 1.0 + rng.random((11, 13))
        dz = box(n, c=c, faces=(ABC, DIRICHLET, NEUMANN, ABC, ABC, ABC), omega=9.0)
        F = dz.load(rng.standard_normal(dz.shape) + 1j * rng.standard_normal(dz.shape),
                    rng.standard_normal(dz.shape) + 0j)
    U = direct.solve(dz, F)
    res = cmcg.solve(dz, F, tol=1e-13)
    assert res.rel_residual <= 1e-13
    assert rel_err(dz, res.u, U) <= 1e-10, case
    # J decreases along CG and vanishes at the solution (Eq. cost_functional_J is zero
    # exactly at the periodic solution).
    J = np.array(res.J_history)
    assert J[-1] <= 1e-20 * J[0]
    assert np.all(np.diff(J) <= 1e-12 * J[0])


# ----------------------------------------------------------------------------------------
# P7 on the functional itself (Eq. cost_functional_J): J = 1/2 ||Pi(v) - v||_E^2 vanishes at
# the periodic state of the direct solve; it is exactly quadratic about that state,
# J(v* + t d) = t^2 J_hom(d); and its central difference along d equals <J'(v), d> with the
# gradient J' = P^T E e - E e of the CMCG Algorithm's step (2).  A dropped 1/2, a mismatch
# taken as Pi(v) + v, a source applied to the homogeneous part or a wrong transpose fails one.
@pytest.mark.parametrize("case", ["2d_mixed_faces", "3d_sphere"])
def test_functional_J(case):
    rng = np.random.default_rng(11)
    if case == "3d_sphere":
        w = wl.sphere_3d(n=8)
        dz = make(w)
        F = dz.load(w.f, w.g)
    else:
        n = (10, 8)
        c = 1.0 + rng.random((9, 11))
        dz = box(n, c=c, faces=(ABC, DIRICHLET, NEUMANN, ABC, ABC, ABC), omega=7.0)
        F = dz.load(rng.standard_normal(dz.shape) + 1j * rng.standard_normal(dz.shape), None)
    U = direct.solve(dz, F)
    v0s, v1s = direct.periodic_state(dz, U)
    J0 = wave.functional_J(dz, 0 * v0s, 0 * v1s, F)
    assert J0 > 0
    assert wave.functional_J(dz, v0s, v1s, F) <= 1e-22 * J0
    d0, d1 = rng.standard_normal(dz.shape) * dz.act, rng.standard_normal(dz.shape) * dz.act
    Jh = wave.functional_J(dz, d0, d1, None)
    for t in (0.5, -2.0):
        assert wave.functional_J(dz, v0s + t * d0, v1s + t * d1, F) == pytest.approx(t * t * Jh, rel=1e-9)
    w0, w1 = rng.standard_normal(dz.shape) * dz.act, rng.standard_normal(dz.shape) * dz.act
    g0, g1, _, _ = cmcg.gradient(dz, w0, w1, F)
    eps = 1e-3
    fd = (wave.functional_J(dz, w0 + eps * d0, w1 + eps * d1, F)
          - wave.functional_J(dz, w0 - eps * d0, w1 - eps * d1, F)) / (2 * eps)
    assert fd == pytest.approx(float(np.sum(g0 * d0) + np.sum(g1 * d1)), rel=1e-8)


# P7b: on a box with absorbing faces only K is singular, and the periodic state is fixed only
# up to a constant displacement (Theorem 1): (Re U, omega_hat Im U) from the direct solve is a
# fixed point of the period map, and so is (Re U + lambda 1, omega_hat Im U) for any real
# lambda, because a constant displacement at rest solves the homogeneous wave equation
# (K 1 = 0, and B acts on velocities).  A constant velocity does not.  A warm start from a
# solution field relies on the first statement.
def test_functional_J_zero_at_the_field_without_lambda():
    w = wl.gaussian_2d(n=12)
    dz = make(w)
    assert not dz.has_dirichlet
    F = dz.load(w.f, None)
    U = direct.solve(dz, F)
    v0s, v1s = direct.periodic_state(dz, U)
    J0 = wave.functional_J(dz, 0 * v0s, 0 * v1s, F)
    assert J0 > 0
    assert wave.functional_J(dz, v0s, v1s, F) <= 1e-22 * J0
    assert wave.functional_J(dz, v0s + 0.37 * dz.act, v1s, F) <= 1e-22 * J0
    # but not a constant velocity: that grows y linearly and breaks periodicity
    assert wave.functional_J(dz, v0s, v1s + 0.37 * dz.act, F) > 1e-6 * J0


# ----------------------------------------------------------------------------------------
# P3: manufactured discrete plane wave U = exp(i kt x) with (2c/h) sin(kt h/2) = wt.
# The time-discrete Helmholtz residual is zero at every interior node (closed form of the
# 5-point dispersion relation), and CMCG given the boundary residual returns U.
def test_manufactured_plane_wave():
    n = (16, 12)
    dz = box(n, omega=6.0, dt_frac=0.4)
    kt = 2.0 / dz.h * math.asin(dz.omega_tilde * dz.h / 2.0)
    U = wl.manufactured_plane_wave_field(n, dz.h, kt)
    A, ia = direct.helmholtz_matrix(dz)
    F = np.zeros(dz.size, dtype=np.complex128)
    F[ia] = A @ U.ravel()[ia]
    F = F.reshape(dz.shape)
    interior = np.zeros(dz.shape, dtype=bool)
    interior[1:-1, 1:-1] = True
    assert np.abs(F[interior]).max() <= 1e-12 * np.abs(F).max()
    res = cmcg.solve(dz, F, tol=1e-13)
    assert rel_err(dz, res.u, U) <= 1e-10


# ----------------------------------------------------------------------------------------
# P6: the compatibility-condition shift is real (Theorem 1: lambda is a real constant), and
# the fundamental-frequency filter (Sec. 2.2, rectangle rule over one period, exact for the
# discrete time-harmonic solution) removes it to the same answer.
def test_lambda_real_and_filter_agrees():
    w = wl.gaussian_2d(n=16)
    c = 1.0 + 0.4 * np.random.default_rng(8).random(w.c.shape)
    dz = Discretization(w.n, w.h, c, w.omega, w.faces, w.dt_target)
    F = dz.load(w.f, None)
    res = cmcg.solve(dz, F, tol=1e-13)
    lam = res.lam
    assert abs(lam) > 1e-8
    assert abs(lam.imag) <= 1e-10 * abs(lam)
    u_filter, shift = cmcg.filtered(dz, res.v0, res.v1, F)
    assert shift == 0.0
    assert rel_err(dz, u_filter, res.u) <= 1e-10


# P13: the physically bounded domain of Sec. 3.5 (pure Neumann, k = pi/4, exact solution
# u = 16 x^2 (x - 1)^2) lifted to 2D.  (a) The discrete solution converges to u at order 2.
# (b) Started from a run-up, the minimiser carries a linear growth eta t (the constant mode
# has no restoring force): the filter alone is then off by a constant, and the discrete
# compatibility condition of Eq. cc_neumann_eta removes it; plain recovery with the
# lambda shift agrees.  Dropping the eta step, or applying it with the wrong sign, fails (b).
def test_pure_neumann_filter_and_eta():
    errs = []
    for n in (16, 32):
        w = wl.neumann_box_2d(n)
        dz = make(w)
        errs.append(rel_err(dz, direct.solve(dz, dz.load(w.f, None)), wl.neumann_box_exact(n)))
    assert 3.6 <= errs[0] / errs[1] <= 4.4, errs
    w = wl.neumann_box_2d(16)
    dz = make(w)
    F = dz.load(w.f, None)
    U = direct.solve(dz, F)
    y0, v0 = wave.long_time(dz, F, 2)
    res = cmcg.solve(dz, F, tol=1e-13, v_init=(y0, v0))
    eta = float(np.sum(dz.M * res.v1) / np.sum(dz.M))
    assert abs(eta) > 1e-2
    assert rel_err(dz, res.u, U) <= 1e-10
    u_f, shift = cmcg.filtered(dz, res.v0, res.v1, F)
    assert abs(shift) > 1e-2
    assert rel_err(dz, u_f, U) <= 1e-10
    assert rel_err(dz, u_f + shift, U) > 1e-2


# ----------------------------------------------------------------------------------------
# P8: continuum check.  With g_S = (d/dn - i k) u_in and no obstacle, u = u_in exactly solves
# the Helmholtz problem of Eq. HE; the discrete solution converges at second order in h
# (dt proportional to h).  Checks M, B, A at faces/corners, the load and the sign conventions.
@pytest.mark.parametrize("dim", [2, 3])
def test_plane_wave_continuum_order(dim):
    errs = []
    grids = [8, 16, 32] if dim == 3 else [16, 32, 64]
    theta = math.radians(135.0)
    dvec = (math.cos(theta), math.sin(theta)) if dim == 2 else (0.5, 0.0, math.sqrt(3.0) / 2.0)
    omega = 2.0 * math.pi * (1.0 if dim == 3 else 2.0)
    for m in grids:
        n = (m,) * dim
        h = 1.0 / m
        faces = (ABC,) * 6
        dz = Discretization(n, h, np.ones(tuple(k + 1 for k in n)), omega, faces, 0.4 * h)
        g = wl.plane_wave_boundary_datum(n, h, omega, 1.0, dvec, faces)
        U = direct.solve(dz, dz.load(None, g))
        xs = wl.coords(n, h)
        uin = np.exp(1j * omega * sum(x * dd for x, dd in zip(xs, dvec))) * np.ones(dz.shape)
        errs.append(rel_err(dz, U, uin))
    rates = [math.log2(errs[i] / errs[i + 1]) for i in range(len(errs) - 1)]
    assert abs(rates[-1] - 2.0) <= 0.2, (errs, rates)


# P9: the paper's recovery u = v0 + (i/omega) v1 differs from the discrete-exact one by
# O((omega dt)^2) -- the Sec. 4.1 observation that CMCG approaches the direct solve as dt -> 0.
def test_paper_recovery_converges_second_order():
    w = wl.gaussian_2d(n=16)
    errs = []
    for frac in (0.4, 0.2, 0.1):
        dz = Discretization(w.n, w.h, w.c, w.omega, w.faces, frac * w.h)
        U = direct.solve(dz, dz.load(w.f, None))
        v0, v1 = direct.periodic_state(dz, U)
        u_paper = v0 + 1j * v1 / dz.omega
        errs.append(rel_err(dz, u_paper, U))
    rates = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert all(abs(r - 2.0) <= 0.2 for r in rates), rates


# ----------------------------------------------------------------------------------------
# P10: the smooth switch-on of Sec. 4.2.3 against its closed form: theta(0) = 0, theta(t_tr) = 1
# with zero slope there, theta'(0) = pi / t_tr (derivative of (2 - s) s with
# s' = pi / (2 t_tr)), strictly increasing on (0, t_tr) and 1 afterwards.  Dropping the
# (2 - s) factor breaks the slope at t_tr; a wrong argument scale breaks theta(t_tr).
def test_theta_tr_closed_form():
    t_tr = 2.7
    eps = 1e-6
    assert wave.theta_tr(0.0, t_tr) == 0.0
    assert abs(wave.theta_tr(t_tr, t_tr) - 1.0) < 1e-15
    assert abs((wave.theta_tr(t_tr, t_tr) - wave.theta_tr(t_tr - eps, t_tr)) / eps) < 1e-5
    assert abs(wave.theta_tr(eps, t_tr) / eps - math.pi / t_tr) < 1e-5
    ts = np.linspace(0.0, t_tr, 200)
    vals = [wave.theta_tr(t, t_tr) for t in ts]
    assert all(b > a for a, b in zip(vals, vals[1:]))
    assert wave.theta_tr(1.5 * t_tr, t_tr) == 1.0


# P11: the do-nothing state of Sec. 4.2 (Eq. AP_SOLUTION) converges to the time-harmonic
# solution (Eq. AP_WAVE_SOLUTION) -- here the direct solve of the same discrete Helmholtz
# system -- on convex domains with absorbing, Neumann and Dirichlet faces.  A wrong forcing
# phase or sign, the continuous omega in place of omega_hat in the recovery, or a missing
# shift removal leaves an error far above the bound.  Without the ramp, l periods from rest
# are the l-fold period map from zero (the load is T-periodic in the global step index).
@pytest.mark.parametrize("faces", [(ABC,) * 4 + (NEUMANN,) * 2, (ABC, NEUMANN, ABC, NEUMANN, NEUMANN, NEUMANN),
                                   (ABC, DIRICHLET, ABC, ABC, NEUMANN, NEUMANN)])
def test_long_time_converges_to_direct(faces):
    w = wl.gaussian_2d(n=20)
    dz = Discretization(w.n, w.h, w.c, w.omega, faces, w.dt_target)
    F = dz.load(w.f, None)
    U = direct.solve(dz, F)
    errs = []
    for ell in (10, 20, 40, 80):
        y, v = wave.long_time(dz, F, ell)
        errs.append(rel_err(dz, cmcg.asymptotic(dz, y, v, F), U))
    assert all(b < a for a, b in zip(errs, errs[1:])), errs
    assert errs[-1] <= 1e-6, errs
    y, v = wave.long_time(dz, F, 3, smooth=False)
    p, q = np.zeros(dz.shape), np.zeros(dz.shape)
    for _ in range(3):
        p, q = wave.period(dz, p, q, F)
    assert np.allclose(y, p, rtol=0, atol=1e-13 * np.abs(p).max())
    assert np.allclose(v, q, rtol=0, atol=1e-13 * np.abs(q).max())


# P12: the ramped run-up trajectory satisfies the three-level leapfrog scheme of Sec. 4.3.1
# (the form the oracle does not run) with the load theta_tr(t_n) F^n at every level n:
#   M (y^{n+1} - 2 y^n + y^{n-1}) / dt^2 + B (y^{n+1} - y^{n-1}) / (2 dt) + K y^n = theta_n F^n.
# A ramp taken at the wrong time level leaves a residual of the size of theta's increment.
def test_ramped_trajectory_is_three_level_leapfrog():
    w = wl.gaussian_2d(n=20)
    dz = make(w)
    F = dz.load(w.f, None)
    _, _, ys = wave.long_time(dz, F, 2, trajectory=True)
    t_tr = 2 * dz.N * dz.dt
    dt = dz.dt
    worst = 0.0
    for n in range(1, len(ys) - 1):
        lhs = dz.M * (ys[n + 1] - 2 * ys[n] + ys[n - 1]) / dt ** 2 + dz.B * (ys[n + 1] - ys[n - 1]) / (2 * dt) + dz.K(ys[n])
        rhs = wave.theta_tr(n * dt, t_tr) * dz.forcing(F, n) * dz.act
        worst = max(worst, float(np.abs((lhs - rhs) * dz.act).max() / np.abs(F).max()))
    assert worst <= 1e-10, worst


# P14: the staggered grid's link mass and difference operator rebuild the stiffness of the
# second-order scheme, G^T W_e G = K (K itself pinned by P5a), with mixed faces, a Dirichlet
# face, an obstacle and in 3D.  A wrong link weight at a face or a missing edge mask fails.
@pytest.mark.parametrize("n,faces,obstacle", [((6, 5), (ABC, NEUMANN, DIRICHLET, ABC, NEUMANN, NEUMANN), False),
                                              ((4, 5, 3), (ABC,) * 6, False),
                                              ((9, 8), (ABC,) * 4 + (NEUMANN,) * 2, True)])
def test_staggered_GtWG_is_K(n, faces, obstacle):
    h = 1.0 / max(n)
    mask = wl.sphere_mask(n, h, (0.5, 0.4, 0.5)[:len(n)], 0.2) if obstacle else None
    dz = box(n, faces=faces, mask=mask)
    st = first_order.Staggered(dz)
    rng = np.random.default_rng(3)
    for _ in range(4):
        y = rng.standard_normal(dz.shape) * dz.act
        a = st.GT([st.We[k] * g for k, g in enumerate(st.G(y))])
        b = dz.K(y)
        assert np.abs(a - b).max() <= 1e-13 * np.abs(b).max()


# P15: on a closed domain (Neumann and Dirichlet faces, no source) the staggered leapfrog
# conserves 1/2 <v^n, v^{n+1}>_M + 1/2 |p^{n+1/2}|^2_{W_e} exactly (sum by parts of the two
# updates), and with absorbing faces that quantity never increases.  A wrong sign or time
# level in either update, or an unbalanced boundary weight, breaks conservation.
@pytest.mark.parametrize("closed", [True, False])
def test_staggered_energy(closed):
    n = (12, 9)
    faces = (NEUMANN, DIRICHLET, NEUMANN, NEUMANN, NEUMANN, NEUMANN) if closed else (ABC, NEUMANN, ABC, ABC, NEUMANN, NEUMANN)
    rng = np.random.default_rng(5)
    c = 1.0 + 0.5 * rng.random((10, 13))
    dz = box(n, c=c, faces=faces, dt_frac=0.3)
    st = first_order.Staggered(dz)
    p = [rng.standard_normal(dz.shape) * st.edge[a] for a in range(2)]
    v = rng.standard_normal(dz.shape) * dz.act
    energies = []
    for k in range(60):
        p1, v1 = st.step(p, v, k)
        energies.append(0.5 * float(np.sum(dz.M * v * v1)) +
                        0.5 * sum(float(np.sum(st.We[a] * p1[a] ** 2)) for a in range(2)))
        p, v = p1, v1
    e = np.array(energies)
    if closed:
        assert np.abs(e - e[0]).max() <= 1e-12 * abs(e[0])
    else:
        assert np.all(np.diff(e) <= 1e-12 * abs(e[0])) and e[-1] < 0.9 * e[0]


# P16: the transposed period is the transpose: <P x, y> = <x, P^T y> in the plain dot product.
@pytest.mark.parametrize("n,faces", [((10, 7), (ABC, NEUMANN, DIRICHLET, ABC, NEUMANN, NEUMANN)),
                                     ((5, 4, 6), (ABC,) * 6)])
def test_staggered_transpose(n, faces):
    rng = np.random.default_rng(6)
    shape = tuple(m + 1 for m in reversed(n))
    dz = box(n, c=1.0 + 0.5 * rng.random(shape), faces=faces, dt_frac=0.2)
    st = first_order.Staggered(dz)
    d = len(n)
    x = ([rng.standard_normal(shape) * st.edge[a] for a in range(d)], rng.standard_normal(shape) * dz.act)
    y = ([rng.standard_normal(shape) * st.edge[a] for a in range(d)], rng.standard_normal(shape) * dz.act)
    px = st.period(*x)
    qy = st.transposed_period(*y)
    lhs = sum(float(np.sum(px[0][a] * y[0][a])) for a in range(d)) + float(np.sum(px[1] * y[1]))
    rhs = sum(float(np.sum(x[0][a] * qy[0][a])) for a in range(d)) + float(np.sum(x[1] * qy[1]))
    assert abs(lhs - rhs) <= 1e-12 * (abs(lhs) + abs(rhs))


# P17: the first-order CMCG fixed point is the direct solve of the SECOND-order time-discrete
# Helmholtz system (K - wt^2 M - i wh B) U = F^ (the substitution in the first_order module
# header), through both the recovery of Eq. mix_solution and the filter of
# Eq. TH_FILTERED_MIXED_SOLUTION; J^ decreases to ~0.  Swapping wt and wh, sampling the source
# at integer steps, or dropping the boundary term of the recovery fails it.
@pytest.mark.parametrize("case", ["gauss2d", "random2d", "sphere3d"])
def test_first_order_matches_second_order_direct(case):
    w = {"gauss2d": lambda: wl.gaussian_2d(n=16), "random2d": lambda: wl.random_2d_instance(2, n=20),
         "sphere3d": lambda: wl.sphere_3d(n=8)}[case]()
    dz = make(w)
    F = dz.load(w.f, w.g)
    U = direct.solve(dz, F)
    res = first_order.solve(dz, F, tol=1e-13)
    assert rel_err(dz, res.u, U) <= 1e-10
    assert rel_err(dz, res.u_filtered, U) <= 1e-10
    assert res.J_history[-1] <= 1e-20 * max(res.J_history[0], 1e-300)


# P18: pure Neumann (Sec. 3.5 lifted to 2D): from a run-up-like start with a constant velocity
# eta (a steady state of the homogeneous first-order system) the minimiser keeps eta; the
# recovery of Eq. mix_solution is then off by i eta / wt, while the filter removes it
# (the proposition of Sec. 3.2).
def test_first_order_pure_neumann_needs_the_filter():
    w = wl.neumann_box_2d(12)
    dz = make(w)
    F = dz.load(w.f, None)
    U = direct.solve(dz, F)
    st = first_order.Staggered(dz)
    s0 = ([np.zeros(dz.shape), np.zeros(dz.shape)], 0.3 * np.ones(dz.shape))
    res = first_order.solve(dz, F, tol=1e-13, s_init=s0)
    assert rel_err(dz, res.u_filtered, U) <= 1e-9
    assert rel_err(dz, res.u, U) > 1e-3
    assert abs(float(np.mean(res.u - U).imag) - 0.3 / dz.omega_tilde) <= 1e-8
    del st


def test_period_rounding_and_cfl():
    # T/dt is an integer: config with omega = 16 pi, dt = h/2, h = 1/128 -> N = 32.
    w = wl.gaussian_2d(n=128)
    dz = Discretization(w.n, w.h, w.c, w.omega, w.faces, w.dt_target)
    assert dz.N == 32 and abs(dz.N * dz.dt - 2 * math.pi / w.omega) < 1e-15
    # 3D sphere recipe: T = 14.2857 h, dt_target = 0.4 h -> N = 36 (independent of n).
    w3 = wl.sphere_3d(n=8)
    assert make(w3).N == 36
    with pytest.raises(ValueError):
        box((8, 8), dt_frac=0.8)


def test_oracle_is_not_imported_by_the_package():
    import pathlib

    pkg = pathlib.Path(__file__).resolve().parents[1] / "paper_1903_12522_gb300"
    for p in pkg.rglob("*.py"):
        src = p.read_text()
        assert "import oracle" not in src and "from oracle" not in src, p
