"""The precision form at scale and the gradient over the 64 parameter points.

Scale: 100 layers, 10,000,000 water-like + 200,000 CO-like lines, 100,000-point
grid, mixed precision (FP32 Voigt and compensated sums, FP64 offsets and
Boltzmann factor), in the launch configuration of the benchmark step (the full
workspace, every layer in one launch), against
  * the FP64 GPU path on every layer at 1,000 random grid points: 100,000
    (layer, point) pairs, 1% of all pairs;
  * the FP64 oracle on 600 random (layer, point) pairs drawn from 12 random
    layers (the oracle needs a pass over all 10.2M lines per layer it visits).
Both at <= 1e-5 relative where sigma > 1e-6 of the layer maximum.

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


def scale_subsets(L, N):
    """1,000 random grid points (all layers) and 600 random (layer, point) pairs
    in 12 random layers, seeded."""
    rng = np.random.default_rng(W.SEED_SUBSET)
    g_sub = np.sort(rng.choice(N, 1000, replace=False))
    lay = np.sort(rng.choice(L, 12, replace=False))
    li = np.repeat(lay, 50)
    gi = rng.integers(0, N, li.size)
    return g_sub, li, gi


def test_scale_precision_form(xs):
    import oracle
    cfg = W.WORKLOADS["scale"]
    nu = W.grid_lognu(cfg["n_grid"])
    P, _ = W.pressure_layers(cfg["n_layers"])
    T = 1300.0 * P ** 0.1
    L, N = P.size, nu.size
    nu_d, T_d, P_d = dev(nu), dev(T), dev(P)
    g_sub, li, gi = scale_subsets(L, N)
    for sp in (W.water_like(cfg["n_water"]), W.co_like(cfg["n_co"])):
        dl = xs.DeviceLines(sp)
        s = xs.xs_compute(dl, nu_d, T_d, P_d, prec=xs.PREC_MIXED).double().cpu().numpy()
        assert np.all(np.isfinite(s)) and np.all(s >= 0)
        floor = 1e-6 * s.max(axis=1, keepdims=True)  # per layer: sigma > 1e-6 max sigma
        # FP64 GPU path at 1,000 grid points, every layer (1% of the pairs)
        s64 = xs.xs_compute(dl, dev(nu[g_sub]), T_d, P_d, prec=xs.PREC_FP64).cpu().numpy()
        got = s[:, g_sub]
        m = s64 > floor
        assert m.sum() > 0.9 * m.size
        assert np.max(np.abs(got[m] - s64[m]) / s64[m]) < 1e-5
        # FP64 oracle at 600 (layer, point) pairs
        lu, li_local = np.unique(li, return_inverse=True)  # the oracle needs only the sampled layers
        want = oracle.xs_points(sp, nu, T[lu], P[lu], li_local, gi)
        m = want > floor[li, 0]
        assert m.sum() > 0.9 * m.size
        assert np.max(np.abs(s[li, gi][m] - want[m]) / want[m]) < 1e-5
        del dl


def test_scale_layer_chunks_give_the_same_bits(xs):
    """A workspace too small for every layer at once makes the library run the
    layers in chunks (with a different split of the line windows across CTAs);
    the result agrees to FP32 rounding of the partial sums."""
    cfg = W.WORKLOADS["scale"]
    nu = W.grid_lognu(cfg["n_grid"])
    P, _ = W.pressure_layers(cfg["n_layers"])
    T_d, P_d, nu_d = dev(1300.0 * P ** 0.1), dev(P), dev(nu)
    dl = xs.DeviceLines(W.co_like(cfg["n_co"]))
    full = xs.xs_compute(dl, nu_d, T_d, P_d, prec=xs.PREC_MIXED)
    need = xs.workspace_bytes(dl.n, nu.size, P.size, xs.PREC_MIXED)
    ws = torch.empty(need // 7, dtype=torch.uint8, device="cuda")
    chunked = xs.xs_compute(dl, nu_d, T_d, P_d, prec=xs.PREC_MIXED, workspace=ws)
    a, b = full.double().cpu().numpy(), chunked.double().cpu().numpy()
    m = a > 1e-6 * a.max(axis=1, keepdims=True)
    assert np.max(np.abs(a[m] - b[m]) / a[m]) < 1e-6


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
