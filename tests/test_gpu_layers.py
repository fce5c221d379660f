"""Per-layer temperatures (the layer-by-layer retrieval of Sec. 6): the gradient
in every T_n, checked (1) on a power-law profile against the composite model's
dlogL/dT0 and dlogL/dalpha by the chain rule, and (2) on a perturbed profile
against Richardson-extrapolated central differences of the FP64 GPU model."""
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
