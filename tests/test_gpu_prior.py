"""The Gaussian-process prior of the layer-by-layer temperatures (Sec. 6.1) on
the GPU against the oracle: log p(T) and its gradient in every T_n and in T0,
with the paper's hyperparameters (a_T = 1e6, tau_P = 10^0.5, eps = 1e-5) on 100
layers, and with others on 1 and 200 layers.  Both sides are FP64; K is
ill-conditioned (condition number up to ~1e7 with eps = 1e-5), so the solutions
agree to about cond x 1e-16: logp to 1e-9 relative, gradients to 1e-6 of their
largest component."""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.mark.parametrize("L,T0,a,tau,eps", [(100, 1300.0, 1e6, 10 ** 0.5, 1e-5), (1, 1250.0, 4e4, 1.0, 1e-3),
                                            (200, 1400.0, 2.5e5, 0.4, 1e-4), (37, 1100.0, 1e6, 10 ** 0.5, 1e-5)])
def test_prior_matches_oracle(L, T0, a, tau, eps):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import oracle
    from paper_2105_14782_gb300 import xs
    p, _ = W.pressure_layers(L)
    rng = np.random.default_rng(93 + L)
    T = 1300.0 * p ** 0.1 + 150.0 * rng.standard_normal(L)
    lp_o, g_o, g0_o = oracle.gp_prior_layers(T, p, T0, a, tau, eps)
    dev = lambda v: torch.as_tensor(np.asarray(v, dtype=np.float64), device="cuda")
    out = xs.gp_prior_layers(dev(T), dev(p), T0, a, tau, eps).cpu().numpy()
    assert out[0] == pytest.approx(lp_o, rel=1e-9)
    gmax = np.abs(g_o).max()
    assert np.max(np.abs(out[1:1 + L] - g_o)) <= 1e-6 * gmax
    assert out[1 + L] == pytest.approx(g0_o, rel=1e-6, abs=1e-6 * gmax)
    # repeated calls give the same bits (fixed-order reductions)
    again = xs.gp_prior_layers(dev(T), dev(p), T0, a, tau, eps).cpu().numpy()
    assert np.array_equal(out, again)
