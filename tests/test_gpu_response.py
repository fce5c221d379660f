"""Response operators on the GPU (Sec. 4, Eq. responsenu) against the oracle:
rotation with limb darkening, Gaussian IP with a radial velocity onto a
different grid, and both adjoints (the transpose against the oracle's dense
matrix, the vsini and RV derivatives against Richardson-extrapolated central
differences of the oracle)."""
import math

import numpy as np
import pytest

import oracle

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


LO, HI, N = 4360.0, 4370.0, 4000
NU = LO * (HI / LO) ** (np.arange(N) / (N - 1))
DV = oracle.C_KMS * math.log(HI / LO) / (N - 1)  # km/s per grid step
rng = np.random.default_rng(41)
CEN = rng.uniform(4361.0, 4369.0, 60)
F0 = 1.0 - sum(0.5 * rng.uniform() * np.exp(-0.5 * ((NU - c) / 0.01) ** 2) for c in CEN)
NU_OUT = np.linspace(4362.0, 4368.0, 1500)
VSINI = (174 + 0.5) * DV  # kernel edges half a grid step from the nearest points
U1, U2, BETA, RV = 0.45, 0.2, 2.6, 11.3


def richardson(f, x, h):
    d1 = (f(x + h) - f(x - h)) / (2 * h)
    d2 = (f(x + h / 2) - f(x - h / 2)) / h
    return (4 * d2 - d1) / 3


def test_rotation_forward_and_adjoint(xs):
    nu = dev(NU)
    F1 = xs.response_rotation(dev(F0), nu, VSINI, U1, U2).cpu().numpy()
    want = oracle.rotation(F0, NU, VSINI, U1, U2)
    np.testing.assert_allclose(F1, want, rtol=1e-12, atol=0)
    g = rng.standard_normal(N)
    gF0, gv = xs.response_rotation_adjoint(dev(g), dev(F0), nu, VSINI, U1, U2)
    A = oracle.response_matrix(NU, NU, lambda v: oracle.rotation_zeta(v / VSINI, U1, U2))
    np.testing.assert_allclose(gF0.cpu().numpy(), A.T @ g, rtol=1e-11, atol=1e-12 * np.abs(A.T @ g).max())
    fd = richardson(lambda v: g @ oracle.rotation(F0, NU, v, U1, U2), VSINI, 1e-4 * VSINI)
    assert gv.item() == pytest.approx(fd, rel=1e-6)


def test_ip_rv_forward_and_adjoint(xs):
    nu, nuo = dev(NU), dev(NU_OUT)
    F = xs.response_ip_rv(dev(F0), nu, nuo, BETA, RV).cpu().numpy()
    want = oracle.ip_rv(F0, NU, NU_OUT, BETA, RV)
    np.testing.assert_allclose(F, want, rtol=1e-12, atol=0)
    g = rng.standard_normal(NU_OUT.size)
    gF1, grv = xs.response_ip_rv_adjoint(dev(g), dev(F0), nu, nuo, BETA, RV)
    A = oracle.response_matrix(NU, NU_OUT, lambda v: oracle.gauss_ip(v, BETA), RV)
    np.testing.assert_allclose(gF1.cpu().numpy(), A.T @ g, rtol=1e-11, atol=1e-12 * np.abs(A.T @ g).max())
    fd = richardson(lambda r: g @ oracle.ip_rv(F0, NU, NU_OUT, BETA, r), RV, 1e-3)
    assert grv.item() == pytest.approx(fd, rel=1e-7)


def test_chain_keeps_a_constant_and_rejects_bad_arguments(xs):
    nu, nuo = dev(NU), dev(NU_OUT)
    c = torch.full((N,), 3.25, dtype=torch.float64, device="cuda")
    F = xs.response_ip_rv(xs.response_rotation(c, nu, 40.0, 0.6, 0.1), nu, nuo, 3.0, -20.0)
    assert torch.allclose(F, torch.full_like(F, 3.25), rtol=1e-11, atol=0)  # Gaussian sums at shifted nodes
    with pytest.raises(xs.XsError):
        xs.response_rotation(c, nu, 0.0)
    with pytest.raises(xs.XsError):
        xs.response_ip_rv(c, nu, nuo, -1.0)
