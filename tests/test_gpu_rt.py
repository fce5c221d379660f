"""GPU parity of optical depth, emission solve, their adjoints, the likelihood
and the composite model (forward + gradient) against the FP64 CPU oracle."""
import math

import numpy as np
import pytest

import oracle
import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def xs():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_2105_14782_gb300 import xs as _xs
    _xs.lib()
    return _xs


def dev(a):
    return torch.as_tensor(np.asarray(a, dtype=np.float64), device="cuda")


def test_tau_layers_matches_oracle(xs):
    rng = np.random.default_rng(1)
    L, N = 9, 777
    s1, s2 = rng.uniform(0, 1e-20, (L, N)), rng.uniform(0, 1e-21, (L, N))
    P, dP = W.pressure_layers(L)
    vmr = np.array([[1e-3] * L, [5e-4] * L])
    want = oracle.tau([s1, s2], vmr, P, dP)
    got = xs.tau_layers([dev(s1), dev(s2)], dev(vmr), dev(P), dev(dP), prec=xs.PREC_FP64).cpu().numpy()
    assert np.allclose(got, want, rtol=1e-14, atol=0)
    got32 = xs.tau_layers([dev(s1).float(), dev(s2).float()], dev(vmr), dev(P), dev(dP), prec=xs.PREC_MIXED)
    want32 = oracle.tau([dev(s1).float().double().cpu().numpy(), dev(s2).float().double().cpu().numpy()], vmr, P, dP)
    assert np.allclose(got32.cpu().numpy(), want32, rtol=1e-14, atol=0)


@pytest.mark.parametrize("L,N", [(1, 5), (100, 3000)])
def test_emission_matches_oracle(xs, L, N):
    rng = np.random.default_rng(L)
    dtau = rng.lognormal(-1.0, 3.0, (L, N))
    dtau[0, : min(3, N)] = [0.0, 1e-12, 800.0][: min(3, N)]
    T = np.linspace(600.0, 2100.0, L)
    nu = W.grid_lognu(N)
    want = oracle.emission(dtau, T, nu)
    got = xs.emission_spectrum(dev(dtau), dev(T), dev(nu)).cpu().numpy()
    assert np.max(np.abs(got - want) / want) < 1e-13


def test_emission_adjoint_matches_central_differences(xs):
    L, N = 12, 40
    rng = np.random.default_rng(4)
    dtau = rng.lognormal(-1.0, 2.0, (L, N))
    T = np.linspace(700.0, 1900.0, L)
    nu = W.grid_lognu(N)
    lam = rng.standard_normal(N)
    g_dtau, g_T = xs.emission_spectrum_adjoint(dev(lam), dev(dtau), dev(T), dev(nu))
    g_dtau, g_T = g_dtau.cpu().numpy(), g_T.cpu().numpy()
    f = lambda d, t: float(np.dot(lam, oracle.emission(d, t, nu)))

    def richardson(fun, x0, h):
        # central differences at h and h/2 combined to O(h^4), so a larger step
        # keeps the rounding of f (~1e5 here) out of a small derivative
        d1 = (fun(x0 + h) - fun(x0 - h)) / (2 * h)
        d2 = (fun(x0 + h / 2) - fun(x0 - h / 2)) / h
        return (4 * d2 - d1) / 3

    for (n, j) in [(0, 0), (5, 17), (11, 39)]:
        def fd_fun(v, n=n, j=j):
            dd = dtau.copy()
            dd[n, j] = v
            return f(dd, T)
        fd = richardson(fd_fun, dtau[n, j], 1e-2 * dtau[n, j])
        assert g_dtau[n, j] == pytest.approx(fd, rel=1e-6, abs=1e-9 * np.abs(g_dtau).max())
    for n in [0, 6, 11]:
        def ft_fun(v, n=n):
            tt = T.copy()
            tt[n] = v
            return f(dtau, tt)
        fd = richardson(ft_fun, T[n], 1e-2 * T[n])
        assert g_T[n] == pytest.approx(fd, rel=1e-6, abs=1e-9 * np.abs(g_T).max())


def test_loglike_and_temperatures(xs):
    rng = np.random.default_rng(2)
    F, d, s = rng.uniform(1, 2, 1000), rng.uniform(1, 2, 1000), rng.uniform(0.01, 0.02, 1000)
    ll, gF = xs.loglike_gauss(dev(F), dev(d), dev(s))
    assert ll.item() == pytest.approx(oracle.loglike(F, d, s), rel=1e-13)
    assert np.allclose(gF.cpu().numpy(), (d - F) / s ** 2, rtol=1e-14)
    P, _ = W.pressure_layers(10)
    T = xs.layer_temperatures(1300.0, 0.1, dev(P)).cpu().numpy()
    assert np.allclose(T, oracle.temperatures(1300.0, 0.1, P), rtol=1e-14)


def small_atmosphere(n_layers=10, n_grid=900, n1=500, n2=120, W_=2.0):
    p, dp = W.pressure_layers(n_layers)
    nu = W.grid_lognu(n_grid, 4363.0, 4367.0)
    sp1 = W.water_like(n1, seed=51, nu_min=4361.0, nu_max=4369.0)
    sp2 = W.co_like(n2, seed=52, n_bands=3, nu_min=4361.0, nu_max=4369.0)
    return W.Atmosphere(species=[sp1, sp2], vmr=[1e-3, 5e-4], nu=nu, p_bar=p, dp_bar=dp, wing_cut=W_)


@pytest.fixture(scope="module")
def problem():
    atm = small_atmosphere()
    theta_star = np.array([1300.0, 0.1, -3.0, math.log10(5e-4), 1.0])
    F_star = oracle.forward(atm, theta_star)
    sig = 0.01 * F_star
    d = F_star + sig * W.std_normal(F_star.size)
    return atm, d, sig


@pytest.mark.parametrize("theta", [[1250.0, 0.12, -2.8, -3.4, 1.3], [1000.0, 0.05, -5.0, -2.0, 0.5],
                                   [1600.0, 0.2, -2.0, -5.0, 2.0]])
def test_model_forward_and_gradient_match_oracle(xs, problem, theta):
    atm, d, sig = problem
    theta = np.array(theta)
    ll_o, g_o, F_o = oracle.logl_grad(atm, theta, d, sig)
    for prec, tol_f, tol_g in ((xs.PREC_FP64, 1e-10, 1e-8), (xs.PREC_MIXED, 1e-6, 1e-4)):
        model = xs.EmissionModel(atm, prec=prec, d_obs=d, sig_obs=sig)
        F = model.forward(theta).cpu().numpy()
        assert np.max(np.abs(F - F_o) / F_o) < tol_f, prec
        ll, g = model.logl_grad(theta)
        # the likelihood of the GPU's own spectrum, and its distance from the oracle's
        # bounded by the spectrum tolerance: |d logL| <= sum |r| |dF|/s + (1/2) sum (dF/s)^2
        assert ll == pytest.approx(oracle.loglike(F, d, sig), rel=1e-12)
        r, e = (d - F_o) / sig, tol_f * F_o / sig
        assert abs(ll - ll_o) <= np.sum(np.abs(r) * e) + 0.5 * np.sum(e * e), (prec, ll, ll_o)
        scale = np.abs(g_o)
        assert np.all(np.abs(g - g_o) <= tol_g * scale + 1e-12 * scale.max()), (prec, g, g_o)


def test_fp64_gradient_matches_central_differences_on_gpu(xs, problem):
    atm, d, sig = problem
    model = xs.EmissionModel(atm, prec=xs.PREC_FP64, d_obs=d, sig_obs=sig)
    theta = np.array([1250.0, 0.12, -2.8, -3.4, 1.3])
    _, g = model.logl_grad(theta)
    dd, ss = torch.as_tensor(d, device="cuda"), torch.as_tensor(sig, device="cuda")

    def ll(t):
        F = model.forward(t)
        return float(xs.loglike_gauss(F, dd, ss)[0].item())

    for i in range(5):
        h = 1e-4 * abs(theta[i])
        tp, tm = theta.copy(), theta.copy()
        tp[i] += h
        tm[i] -= h
        assert g[i] == pytest.approx((ll(tp) - ll(tm)) / (2 * h), rel=2e-5)


def test_autograd_function(xs, problem):
    atm, d, sig = problem
    model = xs.EmissionModel(atm, prec=xs.PREC_MIXED, d_obs=d, sig_obs=sig)
    theta = torch.tensor([1250.0, 0.12, -2.8, -3.4, 1.3], dtype=torch.float64, requires_grad=True)
    ll = xs.log_likelihood(theta, model)
    ll.backward()
    ll2, g2 = model.logl_grad(theta.detach().numpy())
    assert ll.item() == pytest.approx(ll2, rel=1e-12)
    assert np.allclose(theta.grad.numpy(), g2, rtol=1e-12)
