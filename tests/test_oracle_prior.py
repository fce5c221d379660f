"""Pins of the oracle's layer-temperature prior (Sec. 6.1): a library special
case (scipy's multivariate normal), the closed forms of one layer and of a
kernel too short to couple layers (a diagonal K), the normalisation of a
two-layer density by quadrature, and the gradient against central differences."""
import math

import numpy as np
import pytest

import oracle
import workloads as W


def test_matches_scipy_multivariate_normal():
    from scipy.stats import multivariate_normal
    p, _ = W.pressure_layers(30)
    rng = np.random.default_rng(91)
    T = 1300.0 + 200.0 * rng.standard_normal(30)
    lp = np.log10(p)
    for a, tau, eps in ((1e6, 10 ** 0.5, 1e-5), (2.5e4, 0.3, 1e-3)):
        K = a * np.exp(-(lp[:, None] - lp[None, :]) ** 2 / (2 * tau ** 2)) + eps * a * np.eye(30)
        want = multivariate_normal(mean=np.full(30, 1250.0), cov=K).logpdf(T)
        got, _, _ = oracle.gp_prior_layers(T, p, 1250.0, a, tau, eps)
        assert got == pytest.approx(want, rel=1e-9)


def test_single_layer_closed_form():
    v = 4.0e4 * (1.0 + 1e-3)
    lp, g, g0 = oracle.gp_prior_layers([1400.0], [1.0], 1300.0, 4.0e4, 1.0, 1e-3)
    assert lp == pytest.approx(-0.5 * 100.0 ** 2 / v - 0.5 * math.log(2 * math.pi * v), rel=1e-13)
    assert g[0] == pytest.approx(-100.0 / v, rel=1e-13)
    assert g0 == pytest.approx(100.0 / v, rel=1e-13)


def test_short_kernel_is_independent_layers():
    # tau_P far below the layer spacing: K = a (1 + eps) I to below 1e-300
    p, _ = W.pressure_layers(8)
    T = np.linspace(900.0, 1700.0, 8)
    a, eps = 1e5, 1e-2
    v = a * (1 + eps)
    lp, g, g0 = oracle.gp_prior_layers(T, p, 1300.0, a, 1e-3, eps)
    r = T - 1300.0
    assert lp == pytest.approx(np.sum(-0.5 * r ** 2 / v - 0.5 * np.log(2 * np.pi * v)), rel=1e-13)
    np.testing.assert_allclose(g, -r / v, rtol=1e-13)
    assert g0 == pytest.approx(np.sum(r) / v, rel=1e-12, abs=1e-15)


def test_two_layer_density_integrates_to_one():
    from scipy.integrate import dblquad
    p = np.array([0.1, 1.0])
    a, tau, eps = 1.0, 0.7, 0.05
    f = lambda y, x: math.exp(oracle.gp_prior_layers([x, y], p, 0.0, a, tau, eps)[0])
    val, _ = dblquad(f, -8, 8, -8, 8, epsabs=1e-11)
    assert val == pytest.approx(1.0, abs=1e-8)


def test_gradient_against_central_differences():
    p, _ = W.pressure_layers(12)
    rng = np.random.default_rng(92)
    T = 1300.0 + 100.0 * rng.standard_normal(12)
    a, tau, eps = 1e4, 0.8, 1e-2
    lp0, g, g0 = oracle.gp_prior_layers(T, p, 1250.0, a, tau, eps)
    for n in (0, 5, 11):
        h = 1e-2
        e = np.zeros(12)
        e[n] = h
        fd = (oracle.gp_prior_layers(T + e, p, 1250.0, a, tau, eps)[0]
              - oracle.gp_prior_layers(T - e, p, 1250.0, a, tau, eps)[0]) / (2 * h)
        assert g[n] == pytest.approx(fd, rel=1e-7, abs=1e-10)
    fd0 = (oracle.gp_prior_layers(T, p, 1250.0 + 1e-2, a, tau, eps)[0]
           - oracle.gp_prior_layers(T, p, 1250.0 - 1e-2, a, tau, eps)[0]) / 2e-2
    assert g0 == pytest.approx(fd0, rel=1e-7)
