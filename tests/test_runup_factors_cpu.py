"""The batched run-up's source factors (the engine's forced step kernel) against the one-solve
run-up's.  The one-solve run-up evaluates theta_tr(t_n) cos(omega t_n) and theta_tr(t_n)
sin(omega t_n) on the host in FP64 with t_n = n dt, dt = T / N, t_tr = l T (Eq.
transientfunction); the batched kernel uses omega dt = 2 pi / N, so that the phase is
2 pi (n mod N) / N, and the ramp argument pi t_n / (2 t_tr) = pi n / (2 l N), both in FP32.
The identity holds for every n of every run-up length, to FP32 rounding."""
import math

import numpy as np
import pytest


def host_factors(n, N, periods, omega):
    T = 2.0 * math.pi / omega
    dt = T / N
    t = n * dt
    ttr = periods * T
    s = math.sin(0.5 * math.pi * t / ttr)
    th = 1.0 if t >= ttr else (2.0 - s) * s
    return th * math.cos(omega * t), th * math.sin(omega * t)


def batched_factors(n, N, periods):
    k = n % N
    x = np.float32(2.0) * np.float32(k) / np.float32(N)
    cw = np.float32(math.cos(math.pi * float(x)))  # cos(pi x) of the FP32 argument
    sw = np.float32(math.sin(math.pi * float(x)))
    total = periods * N
    r = np.float32(math.sin(math.pi * float(np.float32(0.5) * np.float32(n) / np.float32(total))))
    th = (np.float32(2.0) - r) * r
    return float(th * cw), float(th * sw)


@pytest.mark.parametrize("N,periods,omega", [(32, 5, 16 * math.pi), (36, 178, 2 * math.pi * 17.92),
                                             (57, 40, 80 * math.pi), (26, 354, 2 * math.pi * 11.0)])
def test_batched_runup_factors_match_the_host_ones(N, periods, omega):
    total = periods * N
    worst = 0.0
    for n in list(range(1, min(total, 400))) + list(range(max(1, total - 400), total)):
        hc, hs = host_factors(n, N, periods, omega)
        bc, bs = batched_factors(n, N, periods)
        worst = max(worst, abs(hc - bc), abs(hs - bs))
    # FP32 rounding of the factors (|factor| <= 1), not a phase drift over hundreds of periods
    assert worst <= 4e-7, worst
