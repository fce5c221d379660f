"""Pins of the oracle's line physics, cross-section sum, optical depth,
transmission, Planck source, emission solve and gradient."""
import math

import numpy as np
import pytest
import scipy.integrate as si
import scipy.special as sp

import oracle
import workloads as W
from tests.golden import load

C2 = load("paper_values.txt")["c2"]


def _lines(n=200, seed=7):
    return W.water_like(n, seed)


# ---------------------------------------------------------------- S, beta, gamma

def test_strength_at_reference_temperature_is_S0():
    ln = _lines()
    S, _, _ = oracle.line_params(ln, 296.0, 1.0)
    assert np.allclose(S, np.exp(ln.ln_S0), rtol=1e-13)


def test_strength_temperature_derivative_closed_form():
    """d ln S/dT of Eq. Slog: c2 E/T^2 - q/T - (c2 nu/T^2) e^{-c2 nu/T}/(1 - e^{-c2 nu/T})."""
    ln = _lines(20)
    T, h = 1300.0, 1e-3
    Sp, _, _ = oracle.line_params(ln, T + h, 1.0)
    Sm, _, _ = oracle.line_params(ln, T - h, 1.0)
    num = (np.log(Sp) - np.log(Sm)) / (2 * h)
    e = np.exp(-C2 * ln.nu_hat / T)
    closed = C2 * ln.elower / T ** 2 - ln.q_exponent / T - (C2 * ln.nu_hat / T ** 2) * e / (1 - e)
    assert np.allclose(num, closed, rtol=1e-6, atol=1e-12)


def test_doppler_width_matches_textbook_hwhm():
    """Doppler HWHM = (nu/c) sqrt(2 ln2 k T / m), the textbook form; beta is its sigma."""
    ln = _lines(5)
    T = 1300.0
    _, beta, _ = oracle.line_params(ln, T, 1.0)
    kB, c, mu = 1.380649e-16, 2.99792458e10, 1.66053906660e-24
    hwhm = ln.nu_hat / c * np.sqrt(2 * math.log(2) * kB * T / (ln.mass_amu * mu))
    assert np.allclose(beta * math.sqrt(2 * math.log(2)), hwhm, rtol=1e-14)
    _, beta4, _ = oracle.line_params(ln, 4 * T, 1.0)
    assert np.allclose(beta4, 2 * beta, rtol=1e-14)


def test_pressure_width_scalings():
    ln = _lines(10)
    _, _, g0 = oracle.line_params(ln, 296.0, 1.01325, sb=1.0)
    assert np.allclose(g0, ln.gamma_ref, rtol=1e-14)  # 296 K and 1 atm
    _, _, g1 = oracle.line_params(ln, 592.0, 2 * 1.01325, sb=1.5)
    assert np.allclose(g1, 1.5 * 2 * ln.gamma_ref * 2.0 ** (-ln.n_temp), rtol=1e-13)


# ---------------------------------------------------------------- cross-section

def test_cross_section_brute_force_tiny():
    """3 lines x 32 points: sum of S V written with scipy's wofz."""
    rng = np.random.default_rng(3)
    ln = W.LineList(np.array([4350.02, 4350.31, 4349.9]), np.log(np.array([1e-21, 3e-22, 2e-20])),
                    np.array([100.0, 2500.0, 4000.0]), np.array([0.03, 0.07, 0.05]), np.array([0.5, 0.7, 0.4]), 18.0)
    nu = np.sort(rng.uniform(4349.5, 4350.8, 32))
    T, P, sb, Wc = 1100.0, 0.3, 1.3, 0.5
    got = oracle.xs(ln, nu, [T], [P], sb=sb, wing_cut=Wc)[0]
    S, beta, gam = oracle.line_params(ln, T, P, sb)
    want = np.zeros_like(nu)
    for l in range(3):
        d = nu - ln.nu_hat[l]
        v = sp.wofz((d + 1j * gam[l]) / (math.sqrt(2) * beta[l])).real / (math.sqrt(2 * math.pi) * beta[l])
        want += np.where(np.abs(d) <= Wc, S[l] * v, 0.0)
    assert np.allclose(got, want, rtol=1e-12, atol=0)


def test_integrated_cross_section_equals_strength_sum_minus_wing_loss():
    ln = W.water_like(40, seed=11, nu_min=4364.5, nu_max=4365.5)
    Wc = 2.0
    T, P = 1300.0, 0.1
    nu = np.linspace(4364.5 - Wc - 0.01, 4365.5 + Wc + 0.01, 400001)
    sig = oracle.xs(ln, nu, [T], [P], wing_cut=Wc)[0]
    S, beta, gam = oracle.line_params(ln, T, P)
    loss = 1.0 - 2.0 / math.pi * np.arctan(Wc / gam)  # Lorentz mass outside |dnu| <= W
    assert np.trapezoid(sig, nu) == pytest.approx(np.sum(S * (1 - loss)), rel=2e-6)


def test_wing_cut_includes_the_boundary():
    ln = W.LineList(np.array([4340.0, 4339.999999]), np.log([1e-21, 1e-21]), np.array([0.0, 0.0]),
                    np.array([0.05, 0.05]), np.array([0.5, 0.5]), 18.0)
    nu = np.array([4365.0])
    one = oracle.xs(ln.subset([0]), nu, [1000.0], [1.0], wing_cut=25.0)[0, 0]
    both = oracle.xs(ln, nu, [1000.0], [1.0], wing_cut=25.0)[0, 0]
    assert one > 0 and both == one


def test_point_sampling_matches_full_grid():
    ln = _lines(300)
    nu = W.grid_lognu(257)
    T = np.array([800.0, 1500.0])
    P = np.array([0.01, 3.0])
    full = oracle.xs(ln, nu, T, P)
    li = np.array([0, 1, 1, 0], dtype=np.int32)
    gi = np.array([0, 5, 256, 100])
    assert np.array_equal(oracle.xs_points(ln, nu, T, P, li, gi), full[li, gi])


# ---------------------------------------------------------------- optical depth

def test_optical_depth_scalings():
    L, N = 3, 5
    rng = np.random.default_rng(0)
    s1, s2 = rng.uniform(0, 1e-20, (L, N)), rng.uniform(0, 1e-20, (L, N))
    P, dP = np.array([0.1, 1.0, 10.0]), np.array([0.05, 0.5, 5.0])
    base = oracle.tau([s1, s2], [[1e-3] * L, [5e-4] * L], P, dP, kappa_coef=0.0)
    only1 = oracle.tau([s1], [[1e-3] * L], P, dP, kappa_coef=0.0)
    only2 = oracle.tau([s2], [[5e-4] * L], P, dP, kappa_coef=0.0)
    assert np.allclose(base, only1 + only2, rtol=1e-14)
    assert np.allclose(oracle.tau([s1], [[2e-3] * L], P, dP, g=2e5, kappa_coef=0.0), only1, rtol=1e-14)
    # column of a 1 bar step of pure H2 (mu = 2.016) under g = 1e5: 1e6 / (mu m_u g) molecules cm^-2
    col = oracle.tau([np.ones((1, 1))], [[1.0]], [1.0], [1.0], mu=2.016, kappa_coef=0.0)[0, 0]
    assert col == pytest.approx(1e6 / 1e5 / (2.016 * 1.66053906660e-24), rel=1e-14)
    cont = oracle.tau([np.zeros((L, N))], [[0.0] * L], P, dP, kappa_coef=1e-8)
    assert np.allclose(cont[:, 0], 1e-8 * P * dP * 1e6 / 1e5, rtol=1e-14)


# ---------------------------------------------------------------- transmission

@pytest.mark.parametrize("x", [1e-6, 1e-3, 0.3, 0.999, 1.0, 1.001, 3.0, 30.0, 200.0])
def test_exponential_integrals_match_scipy(x):
    assert oracle.e1(x) == pytest.approx(sp.exp1(x), rel=1e-13)
    assert oracle.e2(x) == pytest.approx(sp.expn(2, x), rel=1e-13)
    assert oracle.e3(x) == pytest.approx(sp.expn(3, x), rel=1e-13)


def test_transmission_forms_agree_and_limit():
    assert oracle.trans(0.0)[0] == 1.0
    x = np.array([0.5, 0.999999, 1.000001, 2.0])
    two_e3 = 2 * sp.expn(3, x)
    assert np.allclose(oracle.trans(x), two_e3, rtol=1e-13)
    # Eq. trans written out with E1 on both sides of the branch point
    alt = (1 - x) * np.exp(-x) + x * x * sp.exp1(x)
    assert np.allclose(oracle.trans(x), alt, rtol=1e-12)


def test_transmission_within_the_papers_AS70_accuracy():
    """The paper states its A&S E1 fit gives T and 1-T within 2e-7 (Sec. 3, App. A)."""
    g = load("paper_values.txt")
    c = load("abramowitz_stegun_e1.txt")
    x = np.logspace(math.log10(g["trans2E3_range_lo"]), math.log10(g["trans2E3_range_hi"]), 2000)
    small = x <= 1
    e1 = np.empty_like(x)
    xs = x[small]
    e1[small] = -np.log(xs) + c["a0"] + xs * (c["a1"] + xs * (c["a2"] + xs * (c["a3"] + xs * (c["a4"] + xs * c["a5"]))))
    xl = x[~small]
    num = xl ** 4 + c["p1"] * xl ** 3 + c["p2"] * xl ** 2 + c["p3"] * xl + c["p4"]
    den = xl ** 4 + c["q1"] * xl ** 3 + c["q2"] * xl ** 2 + c["q3"] * xl + c["q4"]
    e1[~small] = np.exp(-xl) / xl * num / den
    t_fit = (1 - x) * np.exp(-x) + x * x * e1
    assert np.max(np.abs(oracle.trans(x) - t_fit)) < g["trans2E3_abs_err_f32"]


# ---------------------------------------------------------------- Planck + RT

def test_planck_integrates_to_stefan_boltzmann():
    T = 1300.0
    val, _ = si.quad(lambda nu: oracle.planck_pi(nu, T), 1e-6, 60 * T, limit=400, epsrel=1e-12)
    sigma_sb = 5.670374419e-5
    # c2 is the paper's 1.4387773; CODATA hc/k differs by 3e-7, which enters as T^4 -> 4x
    assert val == pytest.approx(sigma_sb * T ** 4, rel=3e-6)


def test_isothermal_atmosphere_radiates_as_blackbody():
    L, N = 7, 9
    nu = W.grid_lognu(N)
    dtau = np.random.default_rng(1).uniform(0, 3, (L, N))
    T = np.full(L, 1111.0)
    F = oracle.emission(dtau, T, nu)
    assert np.allclose(F, [oracle.planck_pi(v, 1111.0) for v in nu], rtol=1e-13)


def test_transparent_atmosphere_shows_the_bottom():
    L, N = 5, 4
    nu = W.grid_lognu(N)
    T = np.linspace(700, 1500, L)
    F = oracle.emission(np.zeros((L, N)), T, nu)
    assert np.allclose(F, [oracle.planck_pi(v, T[-1]) for v in nu], rtol=1e-14)


def test_one_layer_flux():
    nu = W.grid_lognu(3)
    d = np.array([[0.2, 1.5, 7.0]])
    T = np.array([900.0])
    tr = oracle.trans(d[0])
    S = np.array([oracle.planck_pi(v, 900.0) for v in nu])
    assert np.allclose(oracle.emission(d, T, nu), tr * S + (1 - tr) * S, rtol=1e-14)


def test_recurrence_equals_cumulative_product_form():
    L, N = 30, 11
    nu = W.grid_lognu(N)
    dtau = np.random.default_rng(2).lognormal(-2, 2, (L, N))
    T = np.linspace(600, 2000, L)
    assert np.allclose(oracle.emission(dtau, T, nu), oracle.emission_recurrence(dtau, T, nu), rtol=1e-13)


# ---------------------------------------------------------------- gradient

def tiny_atmosphere(n_layers=6, n_grid=48, n1=60, n2=30):
    p, dp = W.pressure_layers(n_layers)
    nu = W.grid_lognu(n_grid, 4364.0, 4366.0)
    sp1 = W.water_like(n1, seed=21, nu_min=4363.5, nu_max=4366.5)
    sp2 = W.co_like(n2, seed=22, n_bands=3, nu_min=4363.5, nu_max=4366.5)
    return W.Atmosphere(species=[sp1, sp2], vmr=[1e-3, 5e-4], nu=nu, p_bar=p, dp_bar=dp, wing_cut=1.0)


def test_forward_mode_gradient_matches_central_differences():
    atm = tiny_atmosphere()
    theta_star = np.array([1300.0, 0.1, -3.0, math.log10(5e-4), 1.0])
    F_star = oracle.forward(atm, theta_star)
    sig = 0.01 * F_star
    d = F_star + sig * W.std_normal(F_star.size)
    theta = np.array([1250.0, 0.12, -2.7, -3.5, 1.4])
    ll, grad, F0 = oracle.logl_grad(atm, theta, d, sig)
    assert np.allclose(F0, oracle.forward(atm, theta), rtol=1e-13)
    assert ll == pytest.approx(oracle.loglike(F0, d, sig), rel=1e-13)
    for i in range(5):
        h = 1e-4 * abs(theta[i])
        tp, tm = theta.copy(), theta.copy()
        tp[i] += h
        tm[i] -= h
        fd = (oracle.loglike(oracle.forward(atm, tp), d, sig) - oracle.loglike(oracle.forward(atm, tm), d, sig)) / (2 * h)
        assert grad[i] == pytest.approx(fd, rel=1e-5, abs=1e-8 * abs(ll))
