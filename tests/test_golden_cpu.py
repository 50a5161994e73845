"""Pins of the CPU oracle to the paper's printed worked examples (tests/golden/*.txt, each
with its section): with the printed parameters, the oracle's discrete solution converges to
the printed exact solution at the scheme's order (2 in h, with dt proportional to h), and the
workload generators use the printed parameters.  The 1D examples are lifted to a strip of
the plane (Neumann on the y-faces, the solution constant in y); a Dirichlet end with a
nonzero value, which the grid solver does not take, becomes an absorbing face carrying the
exact solution's datum (d/dn - i k) u."""
import math
import os

import numpy as np
import pytest

from oracle import direct
from oracle.grid import ABC, NEUMANN, Discretization
from paper_1903_12522_gb300 import workloads as wl

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def fixture(name):
    out = {}
    for line in open(os.path.join(GOLDEN, name)):
        line = line.split("#", 1)[0].strip()
        if line:
            key, value = (x.strip() for x in line.split("=", 1))
            out[key] = value
    return out


def wnorm(dz, a):
    return math.sqrt(float(np.sum(dz.W * dz.act * np.abs(a) ** 2)))


def strip_solution_errors(k, sign, grids):
    """Relative errors of the direct solve against u = sign * exp(i k x) on strips of m x 2
    intervals, h = 1/m: absorbing at x = 0 (with the datum of u) and at x = 1 (where
    u' - i k u = 0, so the datum vanishes), Neumann on the y-faces."""
    errs = []
    faces = (ABC, ABC, NEUMANN, NEUMANN, NEUMANN, NEUMANN)
    for m in grids:
        n = (m, 2)
        h = 1.0 / m
        dz = Discretization(n, h, np.ones((3, m + 1)), k, faces, 0.4 * h)
        g = sign * wl.plane_wave_boundary_datum(n, h, k, 1.0, (1.0, 0.0), faces)
        U = direct.solve(dz, dz.load(None, g))
        u = sign * np.exp(1j * k * wl.coords(n, h)[0]) * np.ones(dz.shape)
        errs.append(wnorm(dz, U - u) / wnorm(dz, u))
    return errs


def test_sec3_4_example_converges_at_second_order():
    fx = fixture("sec3_4_convergence_example.txt")
    assert fx["solution"] == "-exp(i k x)" and float(fx["c"]) == 1.0
    k = float(fx["k_over_pi"]) * math.pi
    grids = [2 ** int(i) for i in fx["h_exponents"].split()]
    assert grids == [8, 16, 32, 64]
    errs = strip_solution_errors(k, -1.0, grids)
    rates = [math.log2(errs[i] / errs[i + 1]) for i in range(len(errs) - 1)]
    assert errs[-1] < 1e-2 and abs(rates[-1] - 2.0) <= 0.1, (errs, rates)


def test_sec4_1_example_converges_at_second_order():
    fx = fixture("sec4_1_semidiscrete_example.txt")
    assert fx["solution"] == "exp(i k x)" and float(fx["c"]) == 1.0
    k = float(fx["k_over_pi"]) * math.pi
    assert float(fx["omega_over_pi"]) * math.pi == k  # omega = k at c = 1
    errs = strip_solution_errors(k, 1.0, [64, 128, 256, 512])
    rates = [math.log2(errs[i] / errs[i + 1]) for i in range(len(errs) - 1)]
    assert errs[-1] < 1e-2 and all(abs(r - 2.0) <= 0.1 for r in rates[1:]), (errs, rates)


def test_sec3_5_example_parameters_and_convergence():
    fx = fixture("sec3_5_bounded_domain_example.txt")
    k = float(fx["k_over_pi"]) * math.pi
    assert float(fx["omega_over_pi"]) * math.pi == k and float(fx["c"]) == 1.0
    # (4 k)^2 is the first nonzero Neumann eigenvalue pi^2 (times the printed factor)
    assert (4.0 * k) ** 2 == pytest.approx(float(fx["first_eigenvalue_over_pi2"]) * math.pi ** 2, rel=1e-15)
    errs = []
    for n in (16, 32, 64):
        w = wl.neumann_box_2d(n)
        assert w.omega == pytest.approx(k, rel=1e-15) and np.all(w.c == 1.0)
        assert all(f == NEUMANN for f in w.faces[:4])
        dz = Discretization(w.n, w.h, w.c, w.omega, w.faces, w.dt_target)
        U = direct.solve(dz, dz.load(w.f, None))
        u = wl.neumann_box_exact(n)
        x = wl.coords(w.n, w.h)[0]
        assert np.allclose(u, 16.0 * x ** 2 * (x - 1.0) ** 2)  # the printed solution
        errs.append(wnorm(dz, U - u) / wnorm(dz, u))
    rates = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert all(abs(r - 2.0) <= 0.1 for r in rates), (errs, rates)


def test_sec4_2_example_parameters_and_boundary_datum():
    fx = fixture("sec4_2_scattering_example.txt")
    k = float(fx["k_over_pi"]) * math.pi
    assert float(fx["omega_over_pi"]) * math.pi == k and float(fx["c"]) == 1.0
    L = float(fx["domain_wavelengths"]) * (2.0 * math.pi / k)  # 10 wavelengths at c = 1
    theta = math.radians(float(fx["theta_degrees"]))
    d = (math.cos(theta), math.sin(theta))
    n = 64
    w = wl.square_obstacle_2d(n=n)
    # the workload is the printed problem rescaled from (0, L)^2 to the unit square
    assert w.omega == pytest.approx(k * L, rel=1e-15) and np.all(w.c == 1.0)
    assert all(f == ABC for f in w.faces[:4])
    x, y = wl.coords(w.n, w.h)
    uin = np.exp(1j * w.omega * (x * d[0] + y * d[1])) * np.ones(w.shape)
    # the printed datum sign * (d/dn - i k) u_in on each face; the total-field reading takes
    # its negative, (d/dn - i k) u_in, so that u = u_in without the obstacle
    sign = float(fx["g_S_sign_as_printed"])
    inner = slice(1, n)  # face nodes off the corners
    for normal, sl in (((-1.0, 0.0), (inner, 0)), ((1.0, 0.0), (inner, n)), ((0.0, -1.0), (0, inner)),
                       ((0.0, 1.0), (n, inner))):
        printed = sign * 1j * w.omega * (d[0] * normal[0] + d[1] * normal[1] - 1.0) * uin[sl]
        assert np.allclose(w.g[sl], -printed, rtol=1e-12, atol=1e-12)
