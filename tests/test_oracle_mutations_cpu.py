"""Mutation checks of the oracle's pins: each test plants one plausible mistake in the oracle
(on the CPU, by replacing one oracle function for the duration of the test) and requires
that the pin written against that mistake fails.  A pin that still passes with the mistake
in place would not be pinning anything.  The last test runs the same pins unmutated."""
import numpy as np
import pytest

import test_oracle_pins as pins
from oracle import direct, wave


def fails(pin, *args):
    with pytest.raises(AssertionError):
        pin(*args)


def test_recovery_with_omega_for_omega_hat_fails_the_J_pin(monkeypatch):
    # v1 = omega Im U instead of omega_hat Im U (the continuous recovery of Sec. 2.1 used in
    # the discrete setting)
    monkeypatch.setattr(direct, "periodic_state",
                        lambda dz, U: (np.real(U) * dz.act, dz.omega * np.imag(U) * dz.act))
    fails(pins.test_functional_J, "2d_mixed_faces")


def test_dropped_half_in_the_energy_fails_the_J_pin(monkeypatch):
    # J = e.E e instead of 1/2 e.E e: the gradient P^T E e - E e no longer matches J's slope
    orig = wave.energy
    monkeypatch.setattr(wave, "energy", lambda dz, e0, e1: 2.0 * orig(dz, e0, e1))
    fails(pins.test_functional_J, "3d_sphere")


def test_swapped_transpose_outputs_fail_the_adjoint_pin(monkeypatch):
    # the cotangents of y and v returned in the wrong order (a transposed operand)
    orig = wave.transposed_period
    monkeypatch.setattr(wave, "transposed_period", lambda dz, a, b: tuple(reversed(orig(dz, a, b))))
    fails(pins.test_adjoint_dot_product, "mixed2d")


def test_transpose_without_damping_fails_the_adjoint_pin(monkeypatch):
    # the transposed period evaluated as if B were zero (the absorbing term dropped)
    orig = wave.transposed_period

    def mutant(dz, a, b):
        saved = dz.B
        dz.B = np.zeros_like(saved)
        try:
            return orig(dz, a, b)
        finally:
            dz.B = saved

    monkeypatch.setattr(wave, "transposed_period", mutant)
    fails(pins.test_adjoint_dot_product, "abc2d")


def test_flipped_damping_sign_fails_the_energy_pin(monkeypatch):
    # the absorbing term with the wrong sign in the step (energy fed in instead of taken out)
    orig = wave.kick_drift_kick

    def mutant(dz, y, v, Fn, Fn1):
        saved = dz.B
        dz.B = -saved
        try:
            return orig(dz, y, v, Fn, Fn1)
        finally:
            dz.B = saved

    monkeypatch.setattr(wave, "kick_drift_kick", mutant)
    fails(pins.test_energy_identity, False)


def test_ramp_without_its_quadratic_factor_fails_the_ramp_pin(monkeypatch):
    # theta = s instead of (2 - s) s: the slope at t_tr no longer vanishes
    import math

    monkeypatch.setattr(wave, "theta_tr",
                        lambda t, t_tr: 1.0 if t >= t_tr else math.sin(0.5 * math.pi * t / t_tr))
    fails(pins.test_theta_tr_closed_form)


def test_boundary_rows_of_K_scaled_fail_the_eigenmode_pin(monkeypatch):
    # a wrong lumped weight on the faces: K's rows at the boundary nodes 10 % too large
    from oracle.grid import Discretization

    orig = Discretization.K

    def mutant(self, y):
        out = orig(self, y)
        face = np.zeros(self.shape, dtype=bool)
        for ax in range(face.ndim):
            idx = [slice(None)] * face.ndim
            idx[ax] = 0
            face[tuple(idx)] = True
            idx[ax] = -1
            face[tuple(idx)] = True
        return np.where(face, 1.1 * out, out)

    monkeypatch.setattr(Discretization, "K", mutant)
    fails(pins.test_K_cosine_eigenmodes, (6, 9), 2)


def test_the_pins_pass_unmutated():
    pins.test_functional_J("2d_mixed_faces")
    pins.test_functional_J("3d_sphere")
    pins.test_adjoint_dot_product("mixed2d")
    pins.test_adjoint_dot_product("abc2d")
    pins.test_energy_identity(False)
    pins.test_theta_tr_closed_form()
    pins.test_K_cosine_eigenmodes((6, 9), 2)
