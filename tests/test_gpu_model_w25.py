"""The composite model (cross-sections of two species, optical depth, emission
solve, Gaussian likelihood and its gradient) at the workloads' wing cut
W = 25 cm^-1, where the packed Lorentz-wing forms carry almost every evaluation.

(1) A 100-layer, full-band atmosphere (1e-3 .. 1e2 bar, 4340-4390 cm^-1) with
    2,500 water-like + 500 CO-like lines and a 2,000-point grid, against the FP64
    oracle (Sec. 3 pipeline, Eqs. lart2E3 and rerr; Eq. crosssec summed over the
    lines; the gradient by the oracle's forward-mode duals, App. D): the spectrum
    element by element (mixed 1e-6, FP64 1e-10), logL, and the gradient (mixed
    1e-4, FP64 1e-8).
(2) The full emission workload (200,000 + 20,000 lines, 20,000 points, 100
    layers): the mixed path against the FP64 GPU path (itself checked against the
    oracle in (1) and in test_gpu_xs.py), spectrum element by element at two
    parameter points and the gradient at one.

logL bound.  With r_j = (d_j - F_j)/s_j and a spectrum error |dF_j| <= eps F_j,
|d logL| <= sum_j |r_j| eps F_j / s_j + (1/2) sum_j (eps F_j / s_j)^2: the test
asserts that bound (derived from Eq. likelihood) instead of a flat tolerance, and
separately that the GPU's logL is the likelihood of its own spectrum to 1e-12."""
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
    m.lib()
    return m


def full_band_atmosphere():
    p, dp = W.pressure_layers(100)
    return W.Atmosphere(species=[W.water_like(2500, seed=81), W.co_like(500, seed=82)], vmr=[1e-3, 5e-4],
                        nu=W.grid_lognu(2000), p_bar=p, dp_bar=dp, wing_cut=25.0)


def loglike_bound(F_ref, d, sig, eps):
    """Largest |logL(F) - logL(F_ref)| over spectra with |F - F_ref| <= eps F_ref."""
    r = (d - F_ref) / sig
    e = eps * F_ref / sig
    return float(np.sum(np.abs(r) * e) + 0.5 * np.sum(e * e))


@pytest.fixture(scope="module")
def w25(xs):
    import oracle
    atm = full_band_atmosphere()
    F = oracle.forward(atm, W.THETA_STAR)
    sig = 0.01 * F
    d = F + sig * W.std_normal(F.size)
    return atm, d, sig


@pytest.mark.parametrize("k", [-1, 17])
def test_model_at_w25_matches_oracle(xs, w25, k):
    import oracle
    atm, d, sig = w25
    theta = W.THETA_STAR if k < 0 else W.theta_points(64)[k]
    ll_o, g_o, F_o = oracle.logl_grad(atm, theta, d, sig)
    lines = None
    for prec, tol_f, tol_g in ((xs.PREC_FP64, 1e-10, 1e-8), (xs.PREC_MIXED, 1e-6, 1e-4)):
        model = xs.EmissionModel(atm, prec=prec, d_obs=d, sig_obs=sig, lines=lines)
        lines = model.species
        Fbuf = torch.empty(d.size, dtype=torch.float64, device="cuda")
        out = model.logl_grad_async(theta, F0=Fbuf).cpu().numpy()
        F = Fbuf.cpu().numpy()
        ll, g = float(out[0]), out[1:]
        rel = np.abs(F - F_o) / F_o
        assert rel.max() < tol_f, (prec, rel.max(), int(rel.argmax()))
        assert ll == pytest.approx(oracle.loglike(F, d, sig), rel=1e-12)
        assert abs(ll - ll_o) <= loglike_bound(F_o, d, sig, tol_f), (prec, ll, ll_o)
        scale = np.abs(g_o)
        assert np.all(np.abs(g - g_o) <= tol_g * scale + 1e-9 * scale.max()), (prec, g, g_o)
        # forward alone gives the same spectrum bits as the forward inside logl_grad
        assert np.array_equal(model.forward(theta).cpu().numpy(), F)


def test_emission_workload_mixed_against_fp64(xs):
    atm = W.emission_case()
    m64 = xs.EmissionModel(atm, prec=xs.PREC_FP64)
    mmx = xs.EmissionModel(atm, prec=xs.PREC_MIXED, lines=m64.species)
    F_star = mmx.forward(W.THETA_STAR).clone()
    sig = 0.01 * F_star
    d = F_star + sig * torch.as_tensor(W.std_normal(F_star.numel()), device="cuda")
    m64.set_observation(d, sig)
    mmx.set_observation(d, sig)
    # spectrum at theta*
    F64 = m64.forward(W.THETA_STAR).cpu().numpy()
    Fmx = mmx.forward(W.THETA_STAR).cpu().numpy()
    assert np.max(np.abs(Fmx - F64) / F64) < 1e-6
    # spectrum and gradient at a parameter point away from theta*
    theta = W.theta_points(64)[9]
    outs = {}
    for name, m in (("fp64", m64), ("mixed", mmx)):
        Fb = torch.empty(atm.nu.size, dtype=torch.float64, device="cuda")
        o = m.logl_grad_async(theta, F0=Fb).cpu().numpy()
        outs[name] = (o, Fb.cpu().numpy())
    (o64, F64), (omx, Fmx) = outs["fp64"], outs["mixed"]
    assert np.max(np.abs(Fmx - F64) / F64) < 1e-6
    dn, sn = d.cpu().numpy(), sig.cpu().numpy()
    assert abs(omx[0] - o64[0]) <= loglike_bound(F64, dn, sn, 1e-6)
    g64, gmx = o64[1:], omx[1:]
    scale = np.abs(g64)
    assert np.all(np.abs(gmx - g64) <= 1e-4 * scale + 1e-9 * scale.max()), (gmx, g64)
