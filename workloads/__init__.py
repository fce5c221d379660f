"""Seeded synthetic inputs shared by the CUDA path, the oracle, the tests and bench.py.

This module holds no arithmetic of the method itself: it only draws line lists,
builds the wavenumber grid and the pressure layers, and names the workload sizes.
Line strengths are drawn as log10 S0 and handed over as ln S0 (a change of log base
of the drawn number, not a physics step).  Everything is float64 numpy.

Line fields follow the HITRAN-style table of Sec. 2.2 (Table 1): centre nu_hat
[cm^-1], ln S0 at T_ref = 296 K [ln(cm/molecule)], lower-state energy E'' [cm^-1],
Lorentz HWHM gamma_ref at 296 K and 1 atm [cm^-1/atm], temperature exponent n.
Lists are returned in draw order (unsorted); sorting by centre belongs to the
consumers.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

NU_MIN = 4340.0
NU_MAX = 4390.0

# Seeds (numpy PCG64 via default_rng): water-like list 0, CO-like list 1,
# observation noise 2, parameter points 3, serving traffic 4, parity subset 5.
SEED_WATER, SEED_CO, SEED_NOISE, SEED_THETA, SEED_SERVE, SEED_SUBSET = 0, 1, 2, 3, 4, 5


@dataclass
class LineList:
    nu_hat: np.ndarray
    ln_S0: np.ndarray
    elower: np.ndarray
    gamma_ref: np.ndarray
    n_temp: np.ndarray
    mass_amu: float
    q_exponent: float = 1.5  # partition-function ratio Q(T)/Q(296) = (T/296)**q_exponent

    @property
    def n(self) -> int:
        return int(self.nu_hat.shape[0])

    def subset(self, idx) -> "LineList":
        return LineList(self.nu_hat[idx].copy(), self.ln_S0[idx].copy(), self.elower[idx].copy(),
                        self.gamma_ref[idx].copy(), self.n_temp[idx].copy(), self.mass_amu, self.q_exponent)

    def arrays(self):
        return (self.nu_hat, self.ln_S0, self.elower, self.gamma_ref, self.n_temp)


def _draw_fields(rng, n, centres=None, nu_min=NU_MIN, nu_max=NU_MAX):
    # draw order: centres, log10 S0, E'', gamma_ref, n
    if centres is None:
        centres = rng.uniform(nu_min, nu_max, n)
    log10_s0 = rng.uniform(-26.0, -20.0, n)
    elower = rng.uniform(0.0, 5000.0, n)
    gamma_ref = rng.uniform(0.02, 0.1, n)
    n_temp = rng.uniform(0.3, 0.8, n)
    return centres, log10_s0 * math.log(10.0), elower, gamma_ref, n_temp


def water_like(n_lines: int, seed: int = SEED_WATER, nu_min=NU_MIN, nu_max=NU_MAX) -> LineList:
    """Centres uniform over the band, the other fields as the single-layer case."""
    rng = np.random.default_rng(seed)
    f = _draw_fields(rng, n_lines, nu_min=nu_min, nu_max=nu_max)
    return LineList(*f, mass_amu=18.0)


def co_like(n_lines: int, seed: int = SEED_CO, n_bands: int = 5,
            nu_min=NU_MIN, nu_max=NU_MAX) -> LineList:
    """n_bands adjacent bands of equal width; inside band b the centres sit on a
    regular comb (spacing = band width / lines per band, offset half a step)."""
    rng = np.random.default_rng(seed)
    per = n_lines // n_bands
    width = (nu_max - nu_min) / n_bands
    step = width / per
    cen = np.concatenate([nu_min + b * width + (np.arange(per) + 0.5) * step for b in range(n_bands)])
    rest = n_lines - cen.size
    if rest:
        cen = np.concatenate([cen, rng.uniform(nu_min, nu_max, rest)])
    f = _draw_fields(rng, cen.size, centres=cen)
    return LineList(*f, mass_amu=28.0)


def grid_lognu(n: int, nu_min=NU_MIN, nu_max=NU_MAX) -> np.ndarray:
    """n points uniform in log(nu), both ends included."""
    if n == 1:
        return np.array([nu_min])
    j = np.arange(n, dtype=np.float64)
    return nu_min * np.exp(j / (n - 1) * math.log(nu_max / nu_min))


def pressure_layers(n_layers: int, log10_top=-3.0, log10_bottom=2.0):
    """Layer pressures log-spaced from top (index 0) to bottom [bar], and each
    layer's pressure thickness: P_n (1 - 10^{-dlog}), i.e. P_n - P_{n-1}
    extended to the top layer with the same log step."""
    if n_layers == 1:
        return np.array([1.0]), np.array([1.0])
    lg = np.linspace(log10_top, log10_bottom, n_layers)
    p = 10.0 ** lg
    dlog = (log10_bottom - log10_top) / (n_layers - 1)
    return p, p * (1.0 - 10.0 ** (-dlog))


def std_normal(n: int, seed: int = SEED_NOISE) -> np.ndarray:
    return np.random.default_rng(seed).standard_normal(n)


def theta_points(n: int = 64, seed: int = SEED_THETA) -> np.ndarray:
    """Rows (T0, alpha, log10 xi_water, log10 xi_co, broadening scale)."""
    rng = np.random.default_rng(seed)
    return np.stack([rng.uniform(1000.0, 1600.0, n), rng.uniform(0.05, 0.2, n),
                     rng.uniform(-5.0, -2.0, n), rng.uniform(-5.0, -2.0, n),
                     rng.uniform(0.5, 2.0, n)], axis=1)


THETA_STAR = np.array([1300.0, 0.1, math.log10(1e-3), math.log10(5e-4), 1.0])


def subset_pairs(n_layers: int, n_grid: int, frac: float, seed: int = SEED_SUBSET):
    """Random (layer, grid index) pairs without replacement, sorted."""
    rng = np.random.default_rng(seed)
    total = n_layers * n_grid
    k = max(1, int(round(frac * total)))
    flat = np.sort(rng.choice(total, size=k, replace=False))
    return flat // n_grid, flat % n_grid


@dataclass
class Atmosphere:
    """Inputs of one emission problem: species line lists, grid, layers."""
    species: list
    vmr: list            # volume mixing ratio per species (same in every layer)
    nu: np.ndarray
    p_bar: np.ndarray
    dp_bar: np.ndarray
    wing_cut: float = 25.0
    kappa_coef: float = 1e-8   # continuum kappa_c = coef * P[bar]  [cm^2/g]
    gravity: float = 1e5         # cm s^-2
    mu: float = 2.313            # mean molecular weight
    extra: dict = field(default_factory=dict)


def single_layer_case(n_lines=2000, n_grid=4096, seed=SEED_WATER):
    """One layer at 1300 K and 1 bar, 2,000 water-like lines, 4,096-point log grid."""
    lines = water_like(n_lines, seed)
    return lines, grid_lognu(n_grid), np.array([1300.0]), np.array([1.0])


def emission_case(n_water=200_000, n_co=20_000, n_grid=20_000, n_layers=100):
    """100 log-spaced layers 1e-3..1e2 bar, water-like + CO-like species, log grid."""
    p, dp = pressure_layers(n_layers)
    return Atmosphere(species=[water_like(n_water), co_like(n_co)], vmr=[1e-3, 5e-4],
                      nu=grid_lognu(n_grid), p_bar=p, dp_bar=dp)


WORKLOADS = {
    "single_layer": dict(n_lines=2000, n_grid=4096, n_layers=1),
    "emission": dict(n_water=200_000, n_co=20_000, n_grid=20_000, n_layers=100),
    "scale": dict(n_water=10_000_000, n_co=200_000, n_grid=100_000, n_layers=100),
}


def serving_requests(n: int, seed: int = SEED_SERVE):
    """Per request: line count log-uniform in [1e3, 1e6], grid size uniform in
    [2000, 50000], layer count uniform in [20, 200]."""
    rng = np.random.default_rng(seed)
    nl = np.round(10 ** rng.uniform(3.0, 6.0, n)).astype(np.int64)
    ng = rng.integers(2000, 50001, n)
    nlay = rng.integers(20, 201, n)
    return nl, ng, nlay


def cia_table(nu, T_grid=None, alpha0=1e-46, seed=SEED_THETA + 10):
    """A smooth synthetic collision-induced absorption table alpha[nT][N] (cm^5)
    on the grid nu, standing in for a HITRAN CIA table: a broad band centred near
    the middle of the grid whose strength grows with temperature."""
    rng = np.random.default_rng(seed)
    T_grid = np.arange(400.0, 3001.0, 200.0) if T_grid is None else np.asarray(T_grid, dtype=np.float64)
    nu = np.asarray(nu, dtype=np.float64)
    c = 0.5 * (nu[0] + nu[-1]) + rng.uniform(-1.0, 1.0)
    width = 4.0 * (nu[-1] - nu[0]) + 1.0
    band = np.exp(-((nu - c) / width) ** 2)
    return T_grid, alpha0 * (T_grid[:, None] / 1000.0) ** 0.8 * band[None, :]
