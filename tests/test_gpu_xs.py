"""GPU parity of the line-sum cross-section (xs_compute) and its adjoint
against the FP64 CPU oracle, called through the C ABI."""
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


def mixed_ok(got, want, rtol=1e-5, floor=1e-6):
    """BASELINE tolerance for the FP32 form: relative 1e-5 where sigma > 1e-6 max."""
    got = np.asarray(got, dtype=np.float64)
    mask = want > floor * want.max()
    rel = np.abs(got[mask] - want[mask]) / want[mask]
    return rel.max(), mask.mean()


def run_both(xs, lines, nu, T, P, sb=1.0, W_=25.0):
    dl = xs.DeviceLines(lines)
    out = {}
    for prec in (xs.PREC_FP64, xs.PREC_MIXED):
        s = xs.xs_compute(dl, dev(nu), dev(T), dev(P), sb, W_, prec)
        out[prec] = s.double().cpu().numpy()
    return out


def test_single_layer_case_full_grid(xs):
    """One layer, 1300 K, 1 bar, 2,000 lines, 4,096-point log grid, W = 25."""
    lines, nu, T, P = W.single_layer_case()
    want = oracle.xs(lines, nu, T, P)
    got = run_both(xs, lines, nu, T, P)
    assert np.max(np.abs(got[xs.PREC_FP64] - want) / want) < 1e-10
    worst, frac = mixed_ok(got[xs.PREC_MIXED][0], want[0])
    assert worst < 1e-5 and frac > 0.99


def test_layers_span_pressure_range_with_ragged_grid(xs):
    """Five layers from 1e-3 to 1e2 bar (a from ~1e-3 to ~1e2), grid of 2,500
    points (two full 1,024-point strips and a ragged one), lines inside and
    outside the grid."""
    lines = W.water_like(3000, seed=41, nu_min=4330.0, nu_max=4400.0)
    nu = W.grid_lognu(2500, 4350.0, 4352.0)
    P = np.array([1e-3, 1e-2, 1.0, 10.0, 100.0])
    T = np.array([650.0, 800.0, 1300.0, 1600.0, 2000.0])
    want = oracle.xs(lines, nu, T, P, wing_cut=3.0)
    got = run_both(xs, lines, nu, T, P, W_=3.0)
    assert np.max(np.abs(got[xs.PREC_FP64] - want) / want) < 1e-10
    for n in range(5):
        worst, frac = mixed_ok(got[xs.PREC_MIXED][n], want[n])
        assert worst < 1e-5, (n, worst)


def test_isolated_low_pressure_lines_through_every_faddeeva_tier(xs):
    """Few, widely spaced lines at 1e-3 bar: every grid point's sigma is one
    line's Gaussian core, transition or wing, so each tier is seen alone."""
    lines = W.LineList(np.array([4350.1, 4350.6, 4351.3]), np.log([1e-21, 1e-22, 1e-20]), np.array([10.0, 2000.0, 400.0]),
                       np.array([0.05, 0.03, 0.08]), np.array([0.5, 0.6, 0.7]), 18.0)
    nu = np.linspace(4349.9, 4351.6, 3001)
    T, P = np.array([700.0, 1300.0]), np.array([1e-3, 3e-2])
    want = oracle.xs(lines, nu, T, P, wing_cut=25.0)
    got = run_both(xs, lines, nu, T, P)
    assert np.max(np.abs(got[xs.PREC_FP64] - want) / want) < 1e-10
    for n in range(2):
        worst, frac = mixed_ok(got[xs.PREC_MIXED][n], want[n], floor=1e-9)
        assert worst < 1e-5, (n, worst)


def test_wing_cut_boundary_and_lines_outside_grid(xs):
    nu = np.array([4360.0, 4365.0, 4370.0])
    lines = W.LineList(np.array([4339.0, 4340.0, 4395.0, 4400.0]), np.log([1e-20] * 4), np.zeros(4),
                       np.full(4, 0.05), np.full(4, 0.5), 18.0)
    want = oracle.xs(lines, nu, [1000.0], [1.0], wing_cut=25.0)
    got = run_both(xs, lines, nu, [1000.0], [1.0])
    assert want[0, 1] > 0 and want[0, 0] > 0  # 4340 at exactly +-25 of 4365 is included
    assert np.allclose(got[xs.PREC_FP64], want, rtol=1e-12, atol=0)
    assert np.allclose(got[xs.PREC_MIXED], want, rtol=1e-5, atol=0)


def test_empty_line_list_and_single_point(xs):
    empty = W.water_like(0)
    got = run_both(xs, empty, np.array([4360.0, 4361.0]), [1000.0], [1.0])
    assert not got[xs.PREC_FP64].any() and not got[xs.PREC_MIXED].any()
    one = W.water_like(1, seed=3)
    nu = np.array([one.nu_hat[0] + 0.01])
    want = oracle.xs(one, nu, [900.0], [0.5])
    got = run_both(xs, one, nu, [900.0], [0.5])
    assert got[xs.PREC_FP64][0, 0] == pytest.approx(want[0, 0], rel=1e-11)
    assert got[xs.PREC_MIXED][0, 0] == pytest.approx(want[0, 0], rel=1e-5)


def test_small_workspace_runs_layers_in_chunks(xs):
    lines = W.water_like(800, seed=5)
    nu = W.grid_lognu(1500)
    P, _ = W.pressure_layers(7)
    T = 1300.0 * P ** 0.1
    dl = xs.DeviceLines(lines)
    for prec in (xs.PREC_FP64, xs.PREC_MIXED):
        full = xs.xs_compute(dl, dev(nu), dev(T), dev(P), prec=prec)
        small = torch.empty(xs.lib().xs_workspace_min_bytes(800, 1500, 7, prec), dtype=torch.uint8, device="cuda")
        chunked = xs.xs_compute(dl, dev(nu), dev(T), dev(P), prec=prec, workspace=small)
        assert torch.allclose(full.double(), chunked.double(), rtol=1e-6 if prec else 1e-13, atol=0)


def test_deterministic_bits(xs):
    lines = W.water_like(5000, seed=8)
    nu = W.grid_lognu(3000)
    T, P = dev([1000.0, 1500.0]), dev([0.1, 10.0])
    dl = xs.DeviceLines(lines)
    for prec in (xs.PREC_FP64, xs.PREC_MIXED):
        a = xs.xs_compute(dl, dev(nu), T, P, prec=prec)
        b = xs.xs_compute(dl, dev(nu), T, P, prec=prec)
        assert torch.equal(a, b)


def test_unsorted_lines_detected(xs):
    v = dev([4350.0, 4351.0, 4350.5])
    assert xs.check_sorted(v) == xs.XS_EUNSORTED
    assert xs.check_sorted(dev([1.0, 1.0, 2.0])) == xs.XS_OK
    assert xs.check_sorted(dev([1.0, 1.0, 2.0]), strict=True) == xs.XS_EUNSORTED


def test_emission_case_sampled_points_both_species(xs):
    """Full-size 100-layer emission case (200,000 + 20,000 lines, 20,000-point
    grid): GPU sigma against the oracle at 120 sampled (layer, point) pairs."""
    atm = W.emission_case()
    T = 1300.0 * atm.p_bar ** 0.1
    li, gi = W.subset_pairs(100, 20_000, 60 / 2e6)
    for sp in atm.species:
        dl = xs.DeviceLines(sp)
        want = oracle.xs_points(sp, atm.nu, T, atm.p_bar, li, gi)
        for prec, tol in ((xs.PREC_FP64, 1e-10), (xs.PREC_MIXED, 1e-5)):
            s = xs.xs_compute(dl, dev(atm.nu), dev(T), dev(atm.p_bar), prec=prec).double().cpu().numpy()
            got = s[li, gi]
            m = want > 1e-6 * want.max()
            assert np.max(np.abs(got[m] - want[m]) / want[m]) < tol, (prec, sp.mass_amu)


def test_adjoint_matches_central_differences(xs):
    """g_T and g_broad against central differences of the FP64 forward."""
    lines = W.water_like(1500, seed=12, nu_min=4355.0, nu_max=4365.0)
    nu = W.grid_lognu(1800, 4358.0, 4362.0)
    P = np.array([1e-3, 0.05, 2.0, 60.0])
    T = np.array([700.0, 950.0, 1400.0, 1900.0])
    lam = np.random.default_rng(0).standard_normal((4, 1800)) * 1e20
    dl = xs.DeviceLines(lines)
    f = lambda Tv, sb: float((xs.xs_compute(dl, dev(nu), dev(Tv), dev(P), sb, 5.0, xs.PREC_FP64).cpu().numpy()
                              * lam).sum())
    for prec, tol in ((xs.PREC_FP64, 1e-6), (xs.PREC_MIXED, 1e-4)):
        gT, gb = xs.xs_compute_adjoint(dl, dev(nu), dev(T), dev(P), dev(lam), 1.2, 5.0, prec)
        gT, gb = gT.cpu().numpy(), gb.cpu().numpy()[0]
        for n in range(4):
            h = 1e-4 * T[n]
            tp, tm = T.copy(), T.copy()
            tp[n] += h
            tm[n] -= h
            fd = (f(tp, 1.2) - f(tm, 1.2)) / (2 * h)
            assert gT[n] == pytest.approx(fd, rel=tol, abs=1e-6 * abs(fd) + 1e-30), (prec, n)
        h = 1.2e-4
        fd = (f(T, 1.2 + h) - f(T, 1.2 - h)) / (2 * h)
        assert gb == pytest.approx(fd, rel=tol), prec
