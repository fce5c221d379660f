"""Pins of the oracle's MODIT (Sec. 2.1.2, Eq. MODIT) against what the
mathematics fixes: a single line on a q node gives back the Voigt profile in q
(Doppler width beta' = R0 beta/nu_hat, Lorentz width gamma' = R0 gamma/nu_hat);
the lineshape distribution keeps each line's strength, q centroid and ln gamma'
centroid; the q-grid integral of sigma is the sum of strengths; and MODIT agrees
with the direct line-by-line sum to the paper's stated ~1% level."""
import math

import numpy as np
import pytest

import oracle
import workloads as W

NU_MIN, NU_MAX, N = 4362.0, 4368.0, 3000


def grid():
    return NU_MIN * (NU_MAX / NU_MIN) ** (np.arange(N) / (N - 1))


def one_line_at(nu0, P):
    l = W.water_like(1, seed=7, nu_min=4364.0, nu_max=4366.0)
    l.nu_hat[:] = nu0
    return l


@pytest.mark.parametrize("P", [1e-3, 1.0])
def test_single_line_on_a_node_is_the_voigt_profile_in_q(P):
    nu = grid()
    j = 1500
    lines = one_line_at(nu[j], P)
    T = 1300.0
    s = oracle.modit(lines, NU_MIN, NU_MAX, N, [T], [P], n_gamma=1, n_fft=8192)[0]
    R0 = (N - 1) / math.log(NU_MAX / NU_MIN)
    S, beta, gam = oracle.line_params(lines, T, P)
    bq, gq = R0 * beta[0] / nu[j], R0 * gam[0] / nu[j]
    d = np.arange(-8, 9, dtype=float)
    V = oracle.faddeeva(np.abs(d) / (math.sqrt(2) * bq), np.full(d.size, gq / (math.sqrt(2) * bq))).real
    V /= math.sqrt(2 * math.pi) * bq
    got = s[j - 8:j + 9] * nu[j - 8:j + 9] / R0  # back to the q-space density
    np.testing.assert_allclose(got, S[0] * V, rtol=2e-8)


def test_lsd_keeps_strength_and_centroids():
    lines = W.water_like(500, seed=8, nu_min=4363.0, nu_max=4367.0)
    T, P = 1100.0, 0.3
    lsd, nodes, bq, R0 = oracle.modit_lsd(lines, NU_MIN, NU_MAX, N, T, P, 1.0, 12, 8192)
    S, beta, gam = oracle.line_params(lines, T, P)
    q = R0 * np.log(np.asarray(lines.nu_hat) / NU_MIN)
    gq = R0 * gam / np.asarray(lines.nu_hat)
    assert lsd.sum() == pytest.approx(S.sum(), rel=1e-13)
    j = np.arange(lsd.shape[1])
    assert (lsd * j).sum() == pytest.approx((S * q).sum(), rel=1e-12)
    assert (lsd.sum(axis=1) * np.log(nodes)).sum() == pytest.approx((S * np.log(gq)).sum(), rel=1e-12)
    assert nodes[0] == pytest.approx(gq.min(), rel=1e-14) and nodes[-1] == pytest.approx(gq.max(), rel=1e-14)


def test_q_integral_is_the_sum_of_strengths():
    # narrow lines far inside the grid: the wings outside it are below 1e-4
    lines = W.water_like(200, seed=9, nu_min=4364.5, nu_max=4365.5)
    s = oracle.modit(lines, NU_MIN, NU_MAX, N, [900.0], [1e-3])[0]
    R0 = (N - 1) / math.log(NU_MAX / NU_MIN)
    S, _, _ = oracle.line_params(lines, 900.0, 1e-3)
    assert (s * grid() / R0).sum() == pytest.approx(S.sum(), rel=1e-4)


@pytest.mark.parametrize("P,worst,typical", [(1e-2, 3e-2, 5e-3), (1.0, 1e-2, 3e-3)])
def test_modit_matches_direct_sum_to_about_one_percent(P, worst, typical):
    """Against the direct sum with no wing cut.  Linear binning of a centre
    between two q nodes shifts the profile by half a node-weighted second
    derivative, a relative error up to ~1/beta'^2 on the flanks of
    Doppler-dominated lines (beta' ~ 5 q steps here): a few percent at
    1e-2 bar, under 1% when pressure broadening dominates."""
    lines = W.water_like(400, seed=10, nu_min=4363.0, nu_max=4367.0)
    nu = grid()
    T = 1300.0
    m = oracle.modit(lines, NU_MIN, NU_MAX, N, [T], [P], n_gamma=16)[0]
    d = oracle.xs(lines, nu, [T], [P], wing_cut=1e4)[0]
    mask = d > 1e-3 * d.max()
    r = np.abs(m[mask] - d[mask]) / d[mask]
    assert r.max() < worst and np.median(r) < typical


def test_image_sum_matches_brute_force():
    M = 4096
    A = oracle.modit_image_sum(M)
    for d in (0, 1, 7, 300, 2047, -2048, -5):
        p = np.arange(-20000, 20001)
        p = p[p != 0]
        brute = np.sum(1.0 / (np.pi * (d + p * M) ** 2)) + 2.0 / (np.pi * M * M * 20000.5)  # + tail beyond |p| = 20000
        assert A[d % M] == pytest.approx(brute, rel=1e-9)
