"""MODIT on the GPU (modit_compute) against the oracle's MODIT (Sec. 2.1.2,
Eq. MODIT) on the same seeded lines: FP64 to 1e-10 of each layer's maximum
(FFT rounding), FP32 to 1e-5 of it, at a small size with lines beyond the grid
edges and at the size of the 220,000-line emission workload."""
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
    return torch.as_tensor(np.asarray(a, dtype=np.float64), device="cuda")


def check(xs, lines, nu_min, nu_max, N, T, P, n_gamma, tol64=1e-10, tol32=1e-5):
    import oracle
    dl = xs.DeviceLines(lines)
    n_fft = xs.modit_fft_length(nu_min, nu_max, N, dl)
    assert n_fft == oracle.modit_fft_length(nu_min, nu_max, N, lines.nu_hat)
    want = oracle.modit(lines, nu_min, nu_max, N, T, P, n_gamma=n_gamma, n_fft=n_fft)
    scale = np.abs(want).max(axis=1, keepdims=True)
    for prec, tol in ((xs.PREC_FP64, tol64), (xs.PREC_MIXED, tol32)):
        got = xs.modit_compute(dl, nu_min, nu_max, N, dev(T), dev(P), n_gamma=n_gamma, prec=prec).double().cpu().numpy()
        err = np.abs(got - want) / scale
        assert err.max() < tol, (prec, err.max())
    return dl, n_fft


def test_small_case_with_lines_beyond_the_grid(xs):
    lines = W.water_like(3000, seed=31, nu_min=4355.0, nu_max=4375.0)
    P = np.array([1e-3, 0.05, 1.0, 30.0])
    T = 1300.0 * P ** 0.1
    check(xs, lines, 4362.0, 4368.0, 3001, T, P, n_gamma=12)


def test_single_gamma_node_and_narrow_band(xs):
    lines = W.co_like(500, seed=32, n_bands=2, nu_min=4364.0, nu_max=4366.0)
    check(xs, lines, 4363.0, 4367.0, 2048, np.array([900.0]), np.array([0.2]), n_gamma=1)


def test_emission_size_three_layers(xs):
    atm = W.emission_case()
    idx = np.array([0, 50, 99])
    P = atm.p_bar[idx]
    T = 1300.0 * P ** 0.1
    nu = atm.nu
    check(xs, atm.species[0], float(nu[0]), float(nu[-1]), nu.size, T, P, n_gamma=16)


def test_deterministic_and_empty(xs):
    lines = W.water_like(800, seed=33, nu_min=4360.0, nu_max=4370.0)
    dl = xs.DeviceLines(lines)
    T, P = dev([1100.0, 1500.0]), dev([0.01, 3.0])
    a = xs.modit_compute(dl, 4361.0, 4369.0, 4000, T, P)
    b = xs.modit_compute(dl, 4361.0, 4369.0, 4000, T, P)
    assert torch.equal(a, b)
    empty = xs.DeviceLines(lines.subset(np.array([], dtype=np.int64)))
    z = xs.modit_compute(empty, 4361.0, 4369.0, 4000, T, P, n_fft=8192)
    assert torch.count_nonzero(z).item() == 0


def test_rejects_bad_arguments(xs):
    import ctypes as C
    lines = xs.DeviceLines(W.water_like(10, seed=34, nu_min=4364.0, nu_max=4366.0))
    s = lines.struct()
    T, P = dev([1000.0]), dev([1.0])
    out = torch.empty(100, dtype=torch.float64, device="cuda")
    ws = torch.empty(1 << 20, dtype=torch.uint8, device="cuda")
    f = xs.lib().modit_compute
    args = lambda nfft, ng: (C.byref(s), 4364.0, 4366.0, 100, xs._dev(T), xs._dev(P), 1, 1.0, ng, nfft, 0,
                             xs._dev(out), xs._dev(ws), ws.numel(), None)
    assert f(*args(1000, 4)) == xs.XS_EINVAL  # not a power of two
    assert f(*args(64, 4)) == xs.XS_EINVAL    # shorter than the grid
    assert f(*args(256, 33)) == xs.XS_EINVAL  # too many gamma nodes
    assert f(*args(1 << 24, 16)) == xs.XS_EINVAL  # workspace too small


def test_adjoint_matches_central_differences_of_the_oracle(xs):
    import oracle
    lines = W.water_like(800, seed=35, nu_min=4360.0, nu_max=4370.0)
    nu_min, nu_max, N = 4362.0, 4368.0, 3001
    P = np.array([0.01, 0.3, 3.0])
    T = np.array([900.0, 1200.0, 1500.0])
    sb, ng = 1.2, 8
    dl = xs.DeviceLines(lines)
    n_fft = xs.modit_fft_length(nu_min, nu_max, N, dl)
    rng = np.random.default_rng(36)
    g = rng.standard_normal((P.size, N)) * 1e20

    def F(Tv, sbv):
        return float(np.sum(g * oracle.modit(lines, nu_min, nu_max, N, Tv, P, sb=sbv, n_gamma=ng, n_fft=n_fft)))

    def rich(f, x, h):
        d1 = (f(x + h) - f(x - h)) / (2 * h)
        d2 = (f(x + h / 2) - f(x - h / 2)) / h
        return (4 * d2 - d1) / 3

    fd_T = []
    for n in range(P.size):
        e = np.zeros(P.size)
        e[n] = 1.0
        fd_T.append(rich(lambda x: F(T + (x - T[n]) * e, sb), T[n], 1e-3))
    fd_b = rich(lambda x: F(T, x), sb, 1e-6)
    res = {}
    for prec in (xs.PREC_FP64, xs.PREC_MIXED):
        gT, gb = xs.modit_compute_adjoint(dl, nu_min, nu_max, N, dev(T), dev(P), dev(g), broad_scale=sb, n_gamma=ng,
                                          n_fft=n_fft, prec=prec)
        res[prec] = (gT.cpu().numpy(), gb.item())
    gT, gb = res[xs.PREC_FP64]
    np.testing.assert_allclose(gT, fd_T, rtol=1e-5)
    assert gb == pytest.approx(fd_b, rel=1e-5)
    gT32, gb32 = res[xs.PREC_MIXED]
    np.testing.assert_allclose(gT32, gT, rtol=1e-3, atol=1e-4 * np.abs(gT).max())
    assert gb32 == pytest.approx(gb, rel=1e-3)


def test_composite_model_with_modit(xs):
    """Emission model whose cross-sections come from MODIT: spectrum and logL
    against the same pipeline assembled from the oracle (MODIT, optical depth,
    emission, likelihood), gradient against its Richardson differences."""
    import math

    import oracle
    p, dp = W.pressure_layers(8)
    nu = W.grid_lognu(1200, 4363.0, 4367.0)
    atm = W.Atmosphere(species=[W.water_like(600, seed=37, nu_min=4361.0, nu_max=4369.0),
                                W.co_like(150, seed=38, n_bands=2, nu_min=4361.0, nu_max=4369.0)],
                       vmr=[1e-3, 5e-4], nu=nu, p_bar=p, dp_bar=dp)
    ng = 8
    m64 = xs.EmissionModel(atm, prec=xs.PREC_FP64, method="modit", n_gamma=ng)
    nfft = [m64._c.n_fft[i] for i in range(2)]

    def oracle_F(theta):
        T = oracle.temperatures(theta[0], theta[1], p)
        sig = [oracle.modit(sp, nu[0], nu[-1], nu.size, T, p, sb=theta[4], n_gamma=ng, n_fft=nf)
               for sp, nf in zip(atm.species, nfft)]
        vmr = np.array([[10.0 ** theta[2 + k]] * p.size for k in range(2)])
        return oracle.emission(oracle.tau(sig, vmr, p, dp), T, nu)

    ts = np.array([1300.0, 0.1, -3.0, math.log10(5e-4), 1.0])
    Fs = oracle_F(ts)
    sig = 0.01 * Fs
    d = Fs + sig * W.std_normal(Fs.size)
    theta = np.array([1250.0, 0.12, -2.8, -3.4, 1.3])
    F_o = oracle_F(theta)
    ll_o = float(oracle.loglike(F_o, d, sig))
    fd = np.empty(5)
    for i in range(5):
        h = 1e-4 * abs(theta[i])
        f = lambda x: float(oracle.loglike(oracle_F(np.concatenate([theta[:i], [x], theta[i + 1:]])), d, sig))
        d1 = (f(theta[i] + h) - f(theta[i] - h)) / (2 * h)
        d2 = (f(theta[i] + h / 2) - f(theta[i] - h / 2)) / h
        fd[i] = (4 * d2 - d1) / 3
    m64.set_observation(d, sig)
    F = m64.forward(theta).cpu().numpy()
    assert np.max(np.abs(F - F_o) / F_o) < 1e-10
    ll, g = m64.logl_grad(theta)
    assert ll == pytest.approx(ll_o, rel=1e-10)
    np.testing.assert_allclose(g, fd, rtol=2e-5, atol=1e-8 * np.abs(fd).max())
    mmx = xs.EmissionModel(atm, prec=xs.PREC_MIXED, method="modit", n_gamma=ng, d_obs=d, sig_obs=sig,
                           lines=m64.species)
    llm, gm = mmx.logl_grad(theta)
    assert llm == pytest.approx(ll_o, rel=1e-4)
    np.testing.assert_allclose(gm, g, rtol=2e-3, atol=1e-4 * np.abs(g).max())
