"""Pins of the oracle's collision-induced absorption (Sec. 2.4, Eq. taucont): over
an isothermal, constant-alpha atmosphere the layer sum approaches the integral
of n1 n2 alpha over height; alpha at a table temperature is that row, linear
between rows and clamped outside; dtau scales with vmr1 vmr2."""
import math

import numpy as np
import pytest

import oracle
import workloads as W

KB, MU_AMU = 1.380649e-16, 1.66053906660e-24


def test_isothermal_column_matches_the_height_integral():
    # hydrostatic isothermal: n(z) = n_b e^{(z_b - z)/H}; the integral of n^2 over
    # height from the bottom level P_b up to P_t is (n_b^2 - n_t^2) H / 2
    L = 2000
    P = np.logspace(-3, 2, L)
    dP = P * (1 - 10 ** (-5.0 / (L - 1)))
    T, g, mu, v1, v2, a = 1500.0, 1e5, 2.313, 0.8, 0.15, 1e-46
    dt = oracle.tau_cia(np.full((2, 1), a), [1000.0, 2000.0], np.full(L, T), P, dP, v1, v2, g, mu)[:, 0]
    H = KB * T / (mu * MU_AMU * g)
    nb, nt = P[-1] * 1e6 / (KB * T), (P[0] - dP[0]) * 1e6 / (KB * T)
    want = v1 * v2 * a * (nb ** 2 - nt ** 2) * H / 2
    assert dt.sum() == pytest.approx(want, rel=3e-3)  # layer sum vs integral, dlnP = 0.006


def test_interpolation_in_temperature():
    nu = np.linspace(4360.0, 4370.0, 7)
    Tg, alpha = W.cia_table(nu)
    P, dP = np.array([1.0, 1.0, 1.0, 1.0]), np.array([0.1, 0.1, 0.1, 0.1])
    T = np.array([Tg[3], 0.5 * (Tg[3] + Tg[4]), Tg[0] - 100.0, Tg[-1] + 100.0])
    dt = oracle.tau_cia(alpha, Tg, T, P, dP, 1.0, 1.0)
    fac = lambda t: (P[0] * 1e6 / (KB * t)) ** 2 * KB * t / (2.313 * MU_AMU * 1e5) * dP[0] / P[0]
    np.testing.assert_allclose(dt[0], alpha[3] * fac(T[0]), rtol=1e-13)
    np.testing.assert_allclose(dt[1], 0.5 * (alpha[3] + alpha[4]) * fac(T[1]), rtol=1e-13)
    np.testing.assert_allclose(dt[2], alpha[0] * fac(T[2]), rtol=1e-13)
    np.testing.assert_allclose(dt[3], alpha[-1] * fac(T[3]), rtol=1e-13)
    dt2 = oracle.tau_cia(alpha, Tg, T, P, dP, 2.0, 3.0)
    np.testing.assert_allclose(dt2, 6.0 * dt, rtol=1e-13)
