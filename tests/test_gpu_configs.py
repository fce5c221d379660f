"""The precision form at scale and the gradient over the 64 parameter points.

Scale: 100 layers, 10,000,000 water-like + 200,000 CO-like lines, 100,000-point
grid, mixed precision (FP32 Voigt and compensated sums, FP64 offsets and
Boltzmann factor) against the FP64 oracle on sampled (layer, point) pairs and
against the FP64 GPU path on every layer at sampled grid points.

Gradient: the 64 parameter points (T0, alpha, log10 VMR of both species,
broadening scale) on a 100-layer, full-band atmosphere with reduced line and
grid counts: the FP64 adjoint against central differences (h = 1e-4 relative)
at every point, the mixed adjoint against the FP64 one at every point, and the
FP64 oracle gradient (forward-mode duals) at four points."""
import math

import numpy as np
import pytest

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
    return torch.as_tensor(np.asarray(a), dtype=torch.float64, device="cuda")


def test_scale_precision_form(xs):
    import oracle
    cfg = W.WORKLOADS["scale"]
    nu = W.grid_lognu(cfg["n_grid"])
    P, _ = W.pressure_layers(cfg["n_layers"])
    T = 1300.0 * P ** 0.1
    L, N = P.size, nu.size
    nu_d, T_d, P_d = dev(nu), dev(T), dev(P)
    rng = np.random.default_rng(W.SEED_SUBSET)
    g_sub = np.sort(rng.choice(N, 48, replace=False))
    li, gi = W.subset_pairs(L, N, 40 / (L * N))
    ws = torch.empty(8 << 30, dtype=torch.uint8, device="cuda")  # forces layer chunks
    for sp in (W.water_like(cfg["n_water"]), W.co_like(cfg["n_co"])):
        dl = xs.DeviceLines(sp)
        s = xs.xs_compute(dl, nu_d, T_d, P_d, prec=xs.PREC_MIXED, workspace=ws).double().cpu().numpy()
        assert np.all(np.isfinite(s)) and np.all(s >= 0)
        floor = 1e-6 * s.max(axis=1, keepdims=True)  # per layer: sigma > 1e-6 max sigma
        # FP64 GPU path at 48 grid points, every layer
        s64 = xs.xs_compute(dl, dev(nu[g_sub]), T_d, P_d, prec=xs.PREC_FP64).cpu().numpy()
        got = s[:, g_sub]
        m = s64 > floor
        assert m.sum() > 0.9 * m.size
        assert np.max(np.abs(got[m] - s64[m]) / s64[m]) < 1e-5
        # FP64 oracle at 40 sampled (layer, point) pairs
        lu, li_local = np.unique(li, return_inverse=True)  # the oracle needs only the sampled layers
        want = oracle.xs_points(sp, nu, T[lu], P[lu], li_local, gi)
        m = want > floor[li, 0]
        assert np.max(np.abs(s[li, gi][m] - want[m]) / want[m]) < 1e-5
        del dl


def gradient_atmosphere():
    p, dp = W.pressure_layers(100)
    return W.Atmosphere(species=[W.water_like(1500, seed=61), W.co_like(300, seed=62)], vmr=[1e-3, 5e-4],
                        nu=W.grid_lognu(1000), p_bar=p, dp_bar=dp)


@pytest.fixture(scope="module")
def grad_problem(xs):
    import oracle
    atm = gradient_atmosphere()
    F = oracle.forward(atm, W.THETA_STAR)
    sig = 0.01 * F
    d = F + sig * W.std_normal(F.size)
    return atm, d, sig


def test_gradient_at_all_64_parameter_points(xs, grad_problem):
    atm, d, sig = grad_problem
    m64 = xs.EmissionModel(atm, prec=xs.PREC_FP64, d_obs=d, sig_obs=sig)
    mmx = xs.EmissionModel(atm, prec=xs.PREC_MIXED, d_obs=d, sig_obs=sig, lines=m64.species)
    dd, ss = dev(d), dev(sig)

    def ll(t):
        return float(xs.loglike_gauss(m64.forward(t), dd, ss)[0].item())

    worst_fd, worst_rich, worst_mx = np.zeros(5), np.zeros(5), np.zeros(5)
    for theta in W.theta_points(64):
        _, g = m64.logl_grad(theta)
        _, gm = mmx.logl_grad(theta)
        fd, fd2 = np.empty(5), np.empty(5)
        for i in range(5):
            for k, hh in enumerate((1e-4, 0.5e-4)):
                h = hh * abs(theta[i])
                tp, tm = theta.copy(), theta.copy()
                tp[i] += h
                tm[i] -= h
                (fd if k == 0 else fd2)[i] = (ll(tp) - ll(tm)) / (2 * h)
        rich = (4.0 * fd2 - fd) / 3.0  # Richardson: removes the h^2 term
        den = np.abs(g) + 1e-6 * np.abs(g).max()
        worst_fd = np.maximum(worst_fd, np.abs(g - fd) / den)
        worst_rich = np.maximum(worst_rich, np.abs(g - rich) / den)
        worst_mx = np.maximum(worst_mx, np.abs(gm - g) / den)
    # central differences at h = 1e-4 carry an O(h^2) truncation error of a few
    # 1e-5 where logL is far from its maximum; the extrapolated ones do not
    assert np.all(worst_fd < 2e-4), worst_fd
    assert np.all(worst_rich < 2e-6), (worst_rich, worst_fd)
    assert np.all(worst_mx < 1e-4), worst_mx


@pytest.mark.parametrize("k", [0, 21, 42, 63])
def test_gradient_against_oracle_at_four_points(xs, grad_problem, k):
    import oracle
    atm, d, sig = grad_problem
    theta = W.theta_points(64)[k]
    ll_o, g_o, _ = oracle.logl_grad(atm, theta, d, sig)
    for prec, tol in ((xs.PREC_FP64, 1e-8), (xs.PREC_MIXED, 1e-4)):
        model = xs.EmissionModel(atm, prec=prec, d_obs=d, sig_obs=sig)
        ll, g = model.logl_grad(theta)
        assert ll == pytest.approx(ll_o, rel=tol)
        scale = np.abs(g_o)
        assert np.all(np.abs(g - g_o) <= tol * scale + 1e-9 * scale.max()), (prec, g, g_o)
