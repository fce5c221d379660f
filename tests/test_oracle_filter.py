"""Pins of the oracle's weak-line pre-filter (App. G): the grey continuum's
contribution peaks where its optical depth crosses one (tau ~ P^2, so the
maximum of exp(-tau) dtau/dlnP is at tau = 1); a line that stays optically thin
peaks where P sigma_centre(P) does; a saturated line peaks at the top and is
kept; the temperature of largest strength is the scan's argmax of S(T)."""
import numpy as np
import pytest

import oracle
import workloads as W

P, DP = W.pressure_layers(100)
T_SCAN = np.arange(500.0, 1701.0, 100.0)


def test_continuum_photosphere_is_at_unit_optical_depth():
    lines = W.water_like(5, seed=72)
    _, _, nc = oracle.contribution_filter(lines, P, DP, T_SCAN, 1e-3, kappa_coef=0.1)
    dtc = oracle.tau([np.zeros((P.size, 1))], np.zeros((1, P.size)), P, DP, 1e5, 2.313, 0.1)[:, 0]
    tau = np.cumsum(dtc)
    assert tau[nc - 1] < 1.0 <= tau[nc + 1]  # the crossing is within a layer of the peak


def test_thin_line_peaks_with_p_sigma_and_saturated_line_at_top():
    lines = W.water_like(2, seed=73)
    lines.ln_S0[:] = np.log([1e-40, 1e-19])  # far too weak to matter / saturated at the top
    keep, nh, nc = oracle.contribution_filter(lines, P, DP, T_SCAN, 1e-3, kappa_coef=0.1)
    S = [oracle.line_params(lines.subset([0]), T, 1.0)[0][0] for T in T_SCAN]
    Ts = T_SCAN[int(np.argmax(S))]
    from scipy.special import erfcx
    ps = []
    for k in range(P.size):
        s, b, g = oracle.line_params(lines.subset([0]), Ts, P[k])
        ps.append(P[k] * s[0] / b[0] * erfcx(g[0] / (np.sqrt(2) * b[0])))
    assert nh[0] == int(np.argmax(ps))
    assert nh[1] == 0 and keep[1]
    assert keep[0] == (nh[0] <= nc + 2)


def test_filter_removes_lines_below_the_continuum_photosphere():
    lines = W.water_like(3000, seed=71)
    keep, nh, nc = oracle.contribution_filter(lines, P, DP, T_SCAN, 1e-3, kappa_coef=0.1)
    assert 0 < keep.sum() < lines.nu_hat.size
    assert np.all(keep == (nh <= nc + 2))
