"""The full model of the paper's fit on the GPU: emission, rigid rotation, Gaussian
IP with radial velocity onto an observed grid, Gaussian likelihood there, and
its gradient in (T0, alpha, log10 VMRs, s_b, vsini, RV) through the responses'
adjoints and the composite model's vector-Jacobian product; against the same
pipeline built from the oracle, and its Richardson-extrapolated differences."""
import math

import numpy as np
import pytest

import oracle
import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def small_atmosphere():
    p, dp = W.pressure_layers(10)
    nu = W.grid_lognu(900, 4363.0, 4367.0)
    sp1 = W.water_like(500, seed=51, nu_min=4361.0, nu_max=4369.0)
    sp2 = W.co_like(120, seed=52, n_bands=3, nu_min=4361.0, nu_max=4369.0)
    return W.Atmosphere(species=[sp1, sp2], vmr=[1e-3, 5e-4], nu=nu, p_bar=p, dp_bar=dp, wing_cut=2.0)


ATM = small_atmosphere()
NU_OBS = np.linspace(4363.6, 4366.4, 300)
BETA, U1, U2 = 3.0, 0.4, 0.2
DV = oracle.C_KMS * math.log(4367.0 / 4363.0) / 899


def oracle_spectrum(theta):
    F0 = oracle.forward(ATM, np.asarray(theta[:5]))
    F1 = oracle.rotation(F0, ATM.nu, theta[5], U1, U2)
    return oracle.ip_rv(F1, ATM.nu, NU_OBS, BETA, theta[6])


THETA_STAR = np.array([1300.0, 0.1, -3.0, math.log10(5e-4), 1.0, 80.5 * DV, 5.0])
F_STAR = oracle_spectrum(THETA_STAR)
SIG = 0.01 * F_STAR
D = F_STAR + SIG * W.std_normal(F_STAR.size)


def oracle_logl(theta):
    return float(oracle.loglike(oracle_spectrum(theta), D, SIG))


@pytest.fixture(scope="module")
def xs():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2105_14782_gb300 import xs as m
    return m


THETA = np.array([1250.0, 0.12, -2.8, -3.4, 1.3, 75.5 * DV, 8.0])


def test_observed_model_logl_and_gradient(xs):
    ll_o = oracle_logl(THETA)
    fd = np.empty(THETA.size)
    for i in range(THETA.size):
        h = 1e-4 * abs(THETA[i])
        f = lambda x: oracle_logl(np.concatenate([THETA[:i], [x], THETA[i + 1:]]))
        d1 = (f(THETA[i] + h) - f(THETA[i] - h)) / (2 * h)
        d2 = (f(THETA[i] + h / 2) - f(THETA[i] - h / 2)) / h
        fd[i] = (4 * d2 - d1) / 3
    res = {}
    for prec in (xs.PREC_FP64, xs.PREC_MIXED):
        om = xs.ObservedModel(xs.EmissionModel(ATM, prec=prec), NU_OBS, D, SIG, BETA, U1, U2)
        res[prec] = om.logl_grad(THETA)
    ll64, g64 = res[xs.PREC_FP64]
    assert ll64 == pytest.approx(ll_o, rel=1e-10)
    np.testing.assert_allclose(g64, fd, rtol=2e-6, atol=1e-9 * np.abs(fd).max())
    llm, gm = res[xs.PREC_MIXED]
    assert llm == pytest.approx(ll_o, rel=1e-5)
    np.testing.assert_allclose(gm, g64, rtol=1e-4, atol=1e-6 * np.abs(g64).max())
