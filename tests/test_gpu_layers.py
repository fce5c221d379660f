"""Per-layer temperatures (the layer-by-layer retrieval of Sec. 6): the gradient
in every T_n, checked (1) on a power-law profile against the composite model's
dlogL/dT0 and dlogL/dalpha by the chain rule, (2) on a perturbed profile
against Richardson-extrapolated central differences of the FP64 GPU model, and
(3) against Richardson-extrapolated central differences of the oracle pipeline
(oracle.xs per species -> oracle.tau -> oracle.emission -> oracle.loglike with an
arbitrary T array), at W = 2 on every layer and at W = 25 on a 100-layer
full-band atmosphere, FP64 and mixed."""
import math

import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def atmosphere():
    p, dp = W.pressure_layers(10)
    nu = W.grid_lognu(900, 4363.0, 4367.0)
    sp1 = W.water_like(500, seed=61, nu_min=4361.0, nu_max=4369.0)
    sp2 = W.co_like(120, seed=62, n_bands=3, nu_min=4361.0, nu_max=4369.0)
    return W.Atmosphere(species=[sp1, sp2], vmr=[1e-3, 5e-4], nu=nu, p_bar=p, dp_bar=dp, wing_cut=2.0)


@pytest.fixture(scope="module")
def setup():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2105_14782_gb300 import xs
    atm = atmosphere()
    m = xs.EmissionModel(atm, prec=xs.PREC_FP64)
    F = m.forward(W.THETA_STAR).cpu().numpy()
    sig = 0.01 * F
    m.set_observation(F + sig * W.std_normal(F.size), sig)
    return xs, atm, m


def test_power_law_profile_matches_the_composite_gradient(setup):
    xs, atm, m = setup
    theta = np.array([1250.0, 0.12, -2.8, -3.4, 1.3])
    ll, g = m.logl_grad(theta)
    T = theta[0] * atm.p_bar ** theta[1]
    ll2, gT, gv, gb = m.logl_grad_layers(T, theta[2:4], theta[4])
    assert ll2 == pytest.approx(ll, rel=1e-13)
    assert np.sum(gT * T / theta[0]) == pytest.approx(g[0], rel=1e-10)
    assert np.sum(gT * T * np.log(atm.p_bar)) == pytest.approx(g[1], rel=1e-10)
    np.testing.assert_allclose(gv, g[2:4], rtol=1e-12)
    assert gb == pytest.approx(g[4], rel=1e-12)


def test_perturbed_profile_against_central_differences(setup):
    xs, atm, m = setup
    rng = np.random.default_rng(63)
    T = 1200.0 * atm.p_bar ** 0.1 * (1.0 + 0.05 * rng.standard_normal(atm.p_bar.size))
    lv, sb = np.array([-3.1, -3.5]), 1.1
    _, gT, _, _ = m.logl_grad_layers(T, lv, sb)

    def ll(Tv):
        return m.logl_grad_layers(Tv, lv, sb)[0]

    for n in (0, 4, 9):
        h = 1e-4 * T[n]
        e = np.zeros_like(T)
        e[n] = 1.0
        d1 = (ll(T + h * e) - ll(T - h * e)) / (2 * h)
        d2 = (ll(T + h / 2 * e) - ll(T - h / 2 * e)) / h
        assert gT[n] == pytest.approx((4 * d2 - d1) / 3, rel=1e-6, abs=1e-9 * np.abs(gT).max())


def oracle_spectrum_layers(atm, T, log10_vmr, sb):
    """F0 of the oracle pipeline with per-layer temperatures T [L]."""
    import oracle
    L = atm.p_bar.size
    sig = [oracle.xs(sp, atm.nu, T, atm.p_bar, sb=sb, wing_cut=atm.wing_cut) for sp in atm.species]
    vmr = np.array([[10.0 ** v] * L for v in log10_vmr])
    dt = oracle.tau(sig, vmr, atm.p_bar, atm.dp_bar, atm.gravity, atm.mu, atm.kappa_coef)
    return oracle.emission(dt, T, atm.nu)


def oracle_loglike_layers(atm, T, log10_vmr, sb, d, s):
    import oracle
    return oracle.loglike(oracle_spectrum_layers(atm, T, log10_vmr, sb), d, s)


def richardson(f, x0, h):
    d1 = (f(x0 + h) - f(x0 - h)) / (2 * h)
    d2 = (f(x0 + h / 2) - f(x0 - h / 2)) / h
    return (4 * d2 - d1) / 3


def full_band_atmosphere():
    p, dp = W.pressure_layers(100)
    return W.Atmosphere(species=[W.water_like(800, seed=64), W.co_like(200, seed=65)], vmr=[1e-3, 5e-4],
                        nu=W.grid_lognu(500), p_bar=p, dp_bar=dp, wing_cut=25.0)


@pytest.mark.parametrize("case", ["w2_all_layers", "w25_100_layers"])
def test_per_layer_gradient_matches_oracle_differences(case):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import oracle
    from paper_2105_14782_gb300 import xs
    atm = atmosphere() if case == "w2_all_layers" else full_band_atmosphere()
    L = atm.p_bar.size
    # observation from the oracle's own forward (seeded noise)
    F = oracle.forward(atm, W.THETA_STAR)
    s = 0.01 * F
    d = F + s * W.std_normal(F.size)
    rng = np.random.default_rng(66)
    T = 1200.0 * atm.p_bar ** 0.1 * (1.0 + 0.05 * rng.standard_normal(L))
    lv, sb = np.array([-3.1, -3.5]), 1.1
    layers = range(L) if L <= 10 else (0, 25, 50, 75, 99)
    fd_T = {}
    for n in layers:
        def f(v, n=n):
            Tv = T.copy()
            Tv[n] = v
            return oracle_loglike_layers(atm, Tv, lv, sb, d, s)
        fd_T[n] = richardson(f, T[n], 1e-4 * T[n])
    fd_v = [richardson(lambda v, m=m: oracle_loglike_layers(atm, T, np.where(np.arange(2) == m, v, lv), sb, d, s),
                       lv[m], 1e-3) for m in range(2)]
    fd_b = richardson(lambda v: oracle_loglike_layers(atm, T, lv, v, d, s), sb, 1e-4 * sb)
    F_T = oracle_spectrum_layers(atm, T, lv, sb)
    ll_o = oracle.loglike(F_T, d, s)
    for prec, tol_f, tol_g in ((xs.PREC_FP64, 1e-10, 1e-6), (xs.PREC_MIXED, 1e-6, 1e-4)):
        m = xs.EmissionModel(atm, prec=prec, d_obs=d, sig_obs=s)
        ll, gT, gv, gb = m.logl_grad_layers(T, lv, sb)
        # |d logL| <= sum |r| |dF|/s + (1/2) sum (dF/s)^2 with |dF| <= tol_f F (Eq. likelihood)
        r, e = (d - F_T) / s, tol_f * F_T / s
        assert abs(ll - ll_o) <= np.sum(np.abs(r) * e) + 0.5 * np.sum(e * e), (prec, ll, ll_o)
        gmax = np.abs(gT).max()
        for n in layers:
            assert gT[n] == pytest.approx(fd_T[n], rel=tol_g, abs=1e-7 * gmax), (prec, n, gT[n], fd_T[n])
        for mm in range(2):
            assert gv[mm] == pytest.approx(fd_v[mm], rel=tol_g), (prec, mm, gv[mm], fd_v[mm])
        assert gb == pytest.approx(fd_b, rel=tol_g), (prec, gb, fd_b)
