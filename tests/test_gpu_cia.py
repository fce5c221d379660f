"""Collision-induced absorption on the GPU (Sec. 2.4, Eq. taucont) against the
oracle: the optical depth, its temperature adjoint (against Richardson
differences of the oracle), and the emission model with the continuum added
(spectrum, logL, gradient)."""
import math

import numpy as np
import pytest

import oracle
import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def xs():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2105_14782_gb300 import xs as m
    return m


def dev(a):
    return torch.as_tensor(np.asarray(a, dtype=np.float64), device="cuda")


def test_tau_cia_and_adjoint(xs):
    p, dp = W.pressure_layers(30)
    nu = W.grid_lognu(500, 4363.0, 4367.0)
    Tg, alpha = W.cia_table(nu)
    T = 1100.0 * p ** 0.12 + 7.3  # off the table's nodes
    want = oracle.tau_cia(alpha, Tg, T, p, dp, 0.84, 0.15)
    got = xs.tau_cia(dev(alpha), dev(Tg), dev(T), dev(p), dev(dp), 0.84, 0.15).cpu().numpy()
    np.testing.assert_allclose(got, want, rtol=1e-13)
    base = dev(np.ones((p.size, nu.size)))
    acc = xs.tau_cia(dev(alpha), dev(Tg), dev(T), dev(p), dev(dp), 0.84, 0.15, out=base).cpu().numpy()
    np.testing.assert_allclose(acc, 1.0 + want, rtol=1e-13)
    g = np.random.default_rng(81).standard_normal((p.size, nu.size))
    gT = xs.tau_cia_adjoint(dev(g), dev(alpha), dev(Tg), dev(T), dev(p), dev(dp), 0.84, 0.15).cpu().numpy()
    for n in (0, 11, 29):
        def f(x):
            Tx = T.copy()
            Tx[n] = x
            return float(np.sum(g * oracle.tau_cia(alpha, Tg, Tx, p, dp, 0.84, 0.15)))
        h = 1e-3
        d1 = (f(T[n] + h) - f(T[n] - h)) / (2 * h)
        d2 = (f(T[n] + h / 2) - f(T[n] - h / 2)) / h
        assert gT[n] == pytest.approx((4 * d2 - d1) / 3, rel=1e-7)


def test_emission_model_with_cia(xs):
    p, dp = W.pressure_layers(10)
    nu = W.grid_lognu(900, 4363.0, 4367.0)
    atm = W.Atmosphere(species=[W.water_like(500, seed=82, nu_min=4361.0, nu_max=4369.0)], vmr=[1e-3], nu=nu,
                       p_bar=p, dp_bar=dp, wing_cut=2.0)
    Tg, alpha = W.cia_table(nu, alpha0=3e-45)
    v1, v2 = 0.84, 0.15

    def oracle_F(theta):
        T = oracle.temperatures(theta[0], theta[1], p)
        sig = oracle.xs(atm.species[0], nu, T, p, sb=theta[3], wing_cut=2.0)
        dt = oracle.tau([sig], np.full((1, p.size), 10.0 ** theta[2]), p, dp) + oracle.tau_cia(alpha, Tg, T, p, dp,
                                                                                               v1, v2)
        return oracle.emission(dt, T, nu)

    ts = np.array([1300.0, 0.1, -3.0, 1.0])
    Fs = oracle_F(ts)
    sig = 0.01 * Fs
    d = Fs + sig * W.std_normal(Fs.size)
    theta = np.array([1250.0, 0.12, -2.8, 1.3])
    m = xs.EmissionModel(atm, prec=xs.PREC_FP64, d_obs=d, sig_obs=sig, cia=(Tg, alpha, v1, v2))
    F = m.forward(theta).cpu().numpy()
    F_o = oracle_F(theta)
    assert np.max(np.abs(F - F_o) / F_o) < 1e-10
    ll, g = m.logl_grad(theta)
    assert ll == pytest.approx(float(oracle.loglike(F_o, d, sig)), rel=1e-10)
    fd = np.empty(4)
    for i in range(4):
        h = 1e-4 * abs(theta[i])
        f = lambda x: float(oracle.loglike(oracle_F(np.concatenate([theta[:i], [x], theta[i + 1:]])), d, sig))
        d1 = (f(theta[i] + h) - f(theta[i] - h)) / (2 * h)
        d2 = (f(theta[i] + h / 2) - f(theta[i] - h / 2)) / h
        fd[i] = (4 * d2 - d1) / 3
    np.testing.assert_allclose(g, fd, rtol=2e-5, atol=1e-8 * np.abs(fd).max())
