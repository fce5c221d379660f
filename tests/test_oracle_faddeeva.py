"""Pins of the oracle's Faddeeva function w(z) = exp(-z^2) erfc(-iz) (Sec. 2.1.1)
against closed forms, library special cases (scipy, mpmath) and the accuracy
the paper states for its own H."""
import math

import numpy as np
import pytest
import scipy.integrate as si
import scipy.special as sp

import oracle
from tests.golden import load

SQRTPI = math.sqrt(math.pi)


def H(x, a):
    return oracle.faddeeva(x, a).real


def test_w_at_origin():
    w = oracle.faddeeva([0.0], [0.0])[0]
    assert w == pytest.approx(1.0, abs=1e-15)


def test_pure_gaussian_limit():
    x = np.linspace(-7.9, 7.9, 301)
    assert np.allclose(H(x, 0.0), np.exp(-x * x), rtol=1e-13, atol=0)
    xb = np.array([8.5, 12.0, 20.0])
    assert np.allclose(H(xb, 0.0), np.exp(-xb * xb), rtol=1e-13, atol=0)


def test_line_centre_is_erfcx():
    a = np.logspace(-4, 3, 71)
    assert np.allclose(H(np.zeros_like(a), a), sp.erfcx(a), rtol=1e-13, atol=0)


def test_matches_scipy_wofz_on_wide_grid():
    xs = np.concatenate([[0.0], np.logspace(-4, 4, 161)])
    as_ = np.logspace(-4, 4, 81)
    X, A = np.meshgrid(xs, as_)
    w = oracle.faddeeva(X.ravel(), A.ravel())
    ref = sp.wofz(X.ravel() + 1j * A.ravel())
    assert np.max(np.abs(w.real - ref.real) / np.abs(ref.real)) < 2e-12
    nz = X.ravel() > 0
    assert np.max(np.abs(w.imag[nz] - ref.imag[nz]) / np.abs(ref.imag[nz])) < 2e-12


def test_negative_x_symmetry():
    x = np.linspace(0.1, 30, 50)
    wp = oracle.faddeeva(x, 0.3)
    wm = oracle.faddeeva(-x, 0.3)
    assert np.allclose(wm, np.conj(wp), rtol=1e-15)


def test_matches_mpmath_in_the_small_a_transition():
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 40
    worst = 0.0
    for x in [0.5, 2.0, 3.0, 4.0, 5.0, 5.9, 7.9, 8.1, 10.0, 30.0, 300.0]:
        for a in [1e-4, 7e-4, 1e-2, 0.3, 2.0, 7.9]:
            z = mp.mpc(x, a)
            ref = complex(mp.exp(-z * z) * mp.erfc(-1j * z))
            w = oracle.faddeeva([x], [a])[0]
            worst = max(worst, abs(w.real - ref.real) / abs(ref.real), abs(w.imag - ref.imag) / abs(ref.imag))
    assert worst < 1e-13


def _hjert_paper(x, a):
    """The paper's H (Sec. 2.1.1): Eq. algo916 with N = 27, eta = 0.5 for
    x^2 + a^2 < 111, Re of the second-order asymptotic form otherwise.
    The sinc arguments follow the series as derived from A&S 7.1.29."""
    g = load("paper_values.txt")
    N, eta = int(g["hjert_N"]), g["hjert_eta"]
    if x * x + a * a >= g["asy_branch_z2"]:
        z = complex(x, a)
        al = 1.0 / (2 * z * z)
        w = 1j / (z * SQRTPI) * (1 + al * (g["asy_s0"] + al * g["asy_s1"]))
        return w.real
    n = np.arange(1, N + 1)
    v0 = 1.0 / (eta ** 2 * n ** 2 + a * a)
    s1 = np.sum(v0 * np.exp(-(eta ** 2 * n ** 2 + x * x)))
    s2 = np.sum(v0 * np.exp(-(eta * n + x) ** 2))
    s3 = np.sum(v0 * np.exp(-(eta * n - x) ** 2))
    sinc = np.sinc(a * x / np.pi)
    return (np.exp(-x * x) * sp.erfcx(a) * np.cos(2 * x * a)
            + 2 * eta * x * np.sin(a * x) / np.pi * np.exp(-x * x) * sinc
            + 2 * eta / np.pi * (-a * np.cos(2 * a * x) * s1 + a / 2 * s2 + a / 2 * s3))


def test_within_the_papers_stated_hjert_accuracy():
    g = load("paper_values.txt")
    worst = 0.0
    for x in np.logspace(-3, 5, 41):
        for a in np.logspace(-3, 5, 21):
            worst = max(worst, abs(H([x], [a])[0] - _hjert_paper(x, a)))
    assert worst < g["hjert_abs_err"]


def test_large_z_approaches_the_papers_asymptotic_series():
    g = load("paper_values.txt")
    s = [g["asy_s0"], g["asy_s1"], g["asy_s2"]]
    for x, a in [(150.0, 0.01), (300.0, 2.0), (120.0, 90.0), (0.0, 200.0)]:
        z = complex(x, a)
        al = 1 / (2 * z * z)
        w_asy = 1j / (z * SQRTPI) * (1 + al * (s[0] + al * (s[1] + al * s[2])))
        w = oracle.faddeeva([x], [a])[0]
        bound = max(105 * abs(al) ** 4 * 10, 1e-14)  # next term of the series (margin 10), or rounding
        assert abs(w - w_asy) / abs(w) < bound


def test_derivative_rules_of_H():
    """dH/dx = 2aL - 2xH and dH/da = 2xL + 2aH - 2/sqrt(pi) (Sec. 2.1.1) by
    central differences of the oracle itself."""
    for x, a in [(0.7, 0.4), (3.0, 0.05), (9.0, 1.5), (40.0, 3.0)]:
        eps = 1e-6 * max(1.0, x)
        w = oracle.faddeeva([x], [a])[0]
        Hx = (H([x + eps], [a])[0] - H([x - eps], [a])[0]) / (2 * eps)
        ea = 1e-6 * max(1.0, a)
        Ha = (H([x], [a + ea])[0] - H([x], [a - ea])[0]) / (2 * ea)
        assert Hx == pytest.approx(2 * a * w.imag - 2 * x * w.real, rel=1e-6, abs=1e-12)
        assert Ha == pytest.approx(2 * x * w.imag + 2 * a * w.real - 2 / SQRTPI, rel=1e-6, abs=1e-12)


def voigt(dnu, beta, gamma):
    s2b = math.sqrt(2) * beta
    return H(np.asarray(dnu) / s2b, gamma / s2b) / (math.sqrt(2 * math.pi) * beta)


@pytest.mark.parametrize("beta,gamma", [(0.011, 0.002), (0.011, 0.05), (0.008, 1e-5)])
def test_voigt_normalisation_within_the_wing_cut(beta, gamma):
    W = 25.0
    x = np.concatenate([np.linspace(-W, -0.5, 200001), np.linspace(-0.5, 0.5, 400001)[1:-1],
                        np.linspace(0.5, W, 200001)])
    inside = np.trapezoid(voigt(x, beta, gamma), x)
    tail = 1.0 - 2.0 / math.pi * math.atan(W / gamma)  # Lorentzian mass beyond |dnu| > W
    assert inside + tail == pytest.approx(1.0, abs=2e-7)


def test_lorentzian_limit():
    gamma = 0.05
    beta = 1e-7
    d = np.array([0.0, 0.01, 0.2, 3.0])
    lor = gamma / (math.pi * (d * d + gamma * gamma))
    assert np.allclose(voigt(d, beta, gamma), lor, rtol=1e-8)


@pytest.mark.parametrize("dnu,beta,gamma", [(0.0, 0.011, 0.03), (0.02, 0.011, 0.001), (0.3, 0.009, 0.08)])
def test_brute_force_convolution(dnu, beta, gamma):
    """V = Gaussian * Lorentzian (the integral form of H, Sec. 2.1.1) by adaptive quadrature."""
    g = lambda t: math.exp(-t * t / (2 * beta * beta)) / (math.sqrt(2 * math.pi) * beta)
    lz = lambda t: gamma / (math.pi * ((dnu - t) ** 2 + gamma ** 2))
    pts = sorted({-10 * beta, 0.0, dnu, 10 * beta})
    val, _ = si.quad(lambda t: g(t) * lz(t), -12 * beta, 12 * beta, points=pts, epsabs=0, epsrel=1e-13, limit=500)
    assert voigt([dnu], beta, gamma)[0] == pytest.approx(val, rel=1e-9)
