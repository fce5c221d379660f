"""Pins of the oracle's response operators (Sec. 4): the rotation kernel against
a direct numerical integral of the limb-darkened disk and against the uniform
disk; its normalisation; Gaussian broadening of a Gaussian line adds variances;
a radial velocity shifts a smooth spectrum; the response keeps a constant."""
import math

import numpy as np
import pytest
from scipy import integrate

import oracle


@pytest.mark.parametrize("u1,u2", [(0.0, 0.0), (0.6, 0.0), (0.4, 0.25), (0.1, 0.7)])
def test_rotation_kernel_is_the_disk_integral(u1, u2):
    def I(y, x):
        mu = math.sqrt(max(0.0, 1.0 - x * x - y * y))
        return 1.0 - u1 * (1.0 - mu) - u2 * (1.0 - mu) ** 2
    tot = integrate.dblquad(I, -1.0, 1.0, lambda x: -math.sqrt(1 - x * x), lambda x: math.sqrt(1 - x * x),
                            epsabs=1e-12, epsrel=1e-12)[0]
    assert tot == pytest.approx(math.pi * (1 - u1 / 3 - u2 / 6), rel=1e-9)
    for x in (0.0, 0.3, -0.55, 0.9, 0.999):
        s = math.sqrt(1 - x * x)
        col = integrate.quad(lambda y: I(y, x), -s, s, epsabs=1e-13, epsrel=1e-12)[0]
        assert oracle.rotation_zeta(x, u1, u2) == pytest.approx(col / tot, rel=1e-9, abs=1e-12)
    assert oracle.rotation_zeta(1.2, u1, u2) == 0.0


def test_uniform_disk_and_normalisation():
    x = np.linspace(-0.99, 0.99, 7)
    np.testing.assert_allclose(oracle.rotation_zeta(x, 0, 0), 2 / np.pi * np.sqrt(1 - x * x), rtol=1e-14)
    assert integrate.quad(lambda t: oracle.rotation_zeta(t, 0.5, 0.2), -1, 1)[0] == pytest.approx(1.0, rel=1e-10)


def log_grid(n, lo=4350.0, hi=4380.0):
    return lo * (hi / lo) ** (np.arange(n) / (n - 1))


def test_gaussian_ip_adds_variances_and_rv_shifts():
    nu = log_grid(6000)
    c = oracle.C_KMS
    v = c * np.log(nu / 4365.0)
    s0, beta = 3.0, 4.0
    F0 = np.exp(-0.5 * (v / s0) ** 2)
    F = oracle.ip_rv(F0, nu, nu, beta, 0.0)
    want = np.exp(-0.5 * v ** 2 / (s0 ** 2 + beta ** 2)) * s0 / math.hypot(s0, beta)
    np.testing.assert_allclose(F, want, atol=2e-4)  # grid quadrature of the convolution
    rv = 7.5
    Fs = oracle.ip_rv(F0, nu, nu, beta, rv)
    # k(c ln(nu'/nu_j) + RV): the profile moves to v' = -RV
    want_s = np.exp(-0.5 * (v + rv) ** 2 / (s0 ** 2 + beta ** 2)) * s0 / math.hypot(s0, beta)
    np.testing.assert_allclose(Fs, want_s, atol=2e-4)


def test_response_keeps_a_constant_away_from_edges():
    nu = log_grid(3000)
    F = oracle.rotation(np.full(nu.size, 2.5), nu, 25.0, 0.4, 0.2)
    np.testing.assert_allclose(F[300:-300], 2.5, rtol=1e-13)
