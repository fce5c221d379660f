"""FP64 CPU oracle (test infrastructure only).

Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg may use this
package.  It wraps the plain C implementation in xs_oracle.c through ctypes; the
C file is compiled here with gcc (OpenMP) on first use or by build().
It shares no code with the CUDA library in paper_2105_14782_gb300/.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "xs_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

_d = C.c_double
_i32 = C.c_int32
_i64 = C.c_int64
_pd = C.POINTER(C.c_double)


def build(force: bool = False) -> str:
    """Compile xs_oracle.c into liboracle.so (gcc -O2 -fopenmp, no fast-math)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.run(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11", _SRC, "-o", tmp, "-lm"],
                       check=True)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = C.CDLL(_LIB)
            lib.orc_num_threads.restype = C.c_int
            lib.orc_faddeeva_v.argtypes = [_i64, _pd, _pd, _pd, _pd]
            lib.orc_line_params.argtypes = [_i64, _pd, _pd, _pd, _pd, _pd, _d, _d, _d, _d, _d, _pd, _pd, _pd]
            lib.orc_xs.argtypes = [_i64, _pd, _pd, _pd, _pd, _pd, _d, _d, _i64, _pd, _i32, _pd, _pd, _d, _d, _pd]
            lib.orc_xs_points.argtypes = [_i64, _pd, _pd, _pd, _pd, _pd, _d, _d, _pd, _i32, _pd, _pd, _d, _d,
                                          _i64, C.POINTER(C.c_int32), C.POINTER(C.c_int64), _pd]
            lib.orc_tau.argtypes = [_i32, C.POINTER(_pd), _pd, _pd, _pd, _i32, _i64, _d, _d, _d, _pd]
            lib.orc_tau_cia.argtypes = [_pd, _pd, _i32, _pd, _pd, _pd, _i32, _i64, _d, _d, _d, _d, _pd]
            for f in ("orc_e1", "orc_e2", "orc_e3", "orc_trans"):
                getattr(lib, f).argtypes = [_d]
                getattr(lib, f).restype = _d
            lib.orc_trans_v.argtypes = [_i64, _pd, _pd]
            lib.orc_planck_pi.argtypes = [_d, _d]
            lib.orc_planck_pi.restype = _d
            lib.orc_emission.argtypes = [_pd, _pd, _pd, _i32, _i64, _pd]
            lib.orc_emission_recurrence.argtypes = [_pd, _pd, _pd, _i32, _i64, _pd]
            lib.orc_loglike.argtypes = [_pd, _pd, _pd, _i64]
            lib.orc_loglike.restype = _d
            lib.orc_logl_grad.argtypes = [_i32, C.POINTER(C.c_int64), _pd, _pd, _pd, _pd, _pd, _pd, _pd, _i64,
                                          _pd, _i32, _pd, _pd, _d, _d, _d, _d, _pd, _pd, _pd, _pd, _pd]
            lib.orc_logl_grad.restype = _d
            _lib = lib
    return _lib


def _p(a):
    return a.ctypes.data_as(_pd)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def num_threads() -> int:
    return int(_load().orc_num_threads())


def faddeeva(x, a):
    """w(x + i a) for a >= 0, elementwise; returns complex128."""
    x = _f64(x).ravel()
    a = _f64(np.broadcast_to(a, x.shape)).ravel()
    re = np.empty_like(x)
    im = np.empty_like(x)
    _load().orc_faddeeva_v(x.size, _p(x), _p(a), _p(re), _p(im))
    return re + 1j * im


def line_params(lines, T, P_bar, sb=1.0):
    """(S(T), beta, gamma) per line, input order."""
    arr = [_f64(v) for v in lines.arrays()]
    n = arr[0].size
    S, b, g = np.empty(n), np.empty(n), np.empty(n)
    _load().orc_line_params(n, *[_p(v) for v in arr], lines.mass_amu, lines.q_exponent, float(T), float(P_bar),
                            float(sb), _p(S), _p(b), _p(g))
    return S, b, g


def xs(lines, nu, T, P_bar, sb=1.0, wing_cut=25.0):
    """sigma[L][N] (cm^2/molecule) for one species."""
    arr = [_f64(v) for v in lines.arrays()]
    nu = _f64(nu)
    T = _f64(np.atleast_1d(T))
    P = _f64(np.atleast_1d(P_bar))
    out = np.empty((T.size, nu.size))
    _load().orc_xs(arr[0].size, *[_p(v) for v in arr], lines.mass_amu, lines.q_exponent, nu.size, _p(nu),
                   T.size, _p(T), _p(P), float(sb), float(wing_cut), _p(out))
    return out


def xs_points(lines, nu, T, P_bar, layer_idx, grid_idx, sb=1.0, wing_cut=25.0):
    """sigma at the given (layer, grid index) pairs."""
    arr = [_f64(v) for v in lines.arrays()]
    nu = _f64(nu)
    T = _f64(np.atleast_1d(T))
    P = _f64(np.atleast_1d(P_bar))
    li = np.ascontiguousarray(layer_idx, dtype=np.int32)
    gi = np.ascontiguousarray(grid_idx, dtype=np.int64)
    out = np.empty(li.size)
    _load().orc_xs_points(arr[0].size, *[_p(v) for v in arr], lines.mass_amu, lines.q_exponent, _p(nu), T.size,
                          _p(T), _p(P), float(sb), float(wing_cut), li.size,
                          li.ctypes.data_as(C.POINTER(C.c_int32)), gi.ctypes.data_as(C.POINTER(C.c_int64)),
                          _p(out))
    return out


def tau(sigmas, vmr, P_bar, dP_bar, g=1e5, mu=2.313, kappa_coef=1e-8):
    """dtau[L][N] from per-species sigma[L][N] and vmr[S][L]."""
    sig = [_f64(s) for s in sigmas]
    L, N = sig[0].shape
    vm = _f64(np.broadcast_to(np.asarray(vmr, dtype=np.float64).reshape(len(sig), -1), (len(sig), L)))
    P, dP = _f64(P_bar), _f64(dP_bar)
    ptrs = (_pd * len(sig))(*[_p(s) for s in sig])
    out = np.empty((L, N))
    _load().orc_tau(len(sig), ptrs, _p(vm), _p(P), _p(dP), L, N, g, mu, kappa_coef, _p(out))
    return out


def tau_cia(alpha, T_grid, T, P_bar, dP_bar, vmr1, vmr2, g=1e5, mu=2.313):
    """dtau[L][N] of a collision-induced absorption pair (Sec. 2.4, Eq. taucont) from the
    table alpha[nT][N] (cm^5) on the model grid, linear in T between T_grid (clamped)."""
    alpha = _f64(alpha)
    Tg, T, P, dP = _f64(T_grid), _f64(np.atleast_1d(T)), _f64(P_bar), _f64(dP_bar)
    nT, N = alpha.shape
    out = np.empty((T.size, N))
    _load().orc_tau_cia(_p(alpha), _p(Tg), nT, _p(T), _p(P), _p(dP), T.size, N, float(vmr1), float(vmr2),
                        float(g), float(mu), _p(out))
    return out


def e1(x):
    return _load().orc_e1(float(x))


def e2(x):
    return _load().orc_e2(float(x))


def e3(x):
    return _load().orc_e3(float(x))


def trans(x):
    x = _f64(np.atleast_1d(x)).ravel()
    out = np.empty_like(x)
    _load().orc_trans_v(x.size, _p(x), _p(out))
    return out


def planck_pi(nu, T):
    return _load().orc_planck_pi(float(nu), float(T))


def emission(dtau, T, nu):
    dtau, T, nu = _f64(dtau), _f64(T), _f64(nu)
    L, N = dtau.shape
    out = np.empty(N)
    _load().orc_emission(_p(dtau), _p(T), _p(nu), L, N, _p(out))
    return out


def emission_recurrence(dtau, T, nu):
    dtau, T, nu = _f64(dtau), _f64(T), _f64(nu)
    L, N = dtau.shape
    out = np.empty(N)
    _load().orc_emission_recurrence(_p(dtau), _p(T), _p(nu), L, N, _p(out))
    return out


def loglike(F, d, sig):
    F, d, sig = _f64(F), _f64(d), _f64(sig)
    return _load().orc_loglike(_p(F), _p(d), _p(sig), F.size)


def temperatures(T0, alpha, P_bar):
    """T_n = T0 (P_n / 1 bar)^alpha (the power-law profile of Sec. 5.2)."""
    return T0 * np.power(_f64(P_bar), alpha)


def forward(atm, theta):
    """F0[N] for theta = (T0, alpha, log10 xi_0..log10 xi_{S-1}, s_b)."""
    S = len(atm.species)
    T = temperatures(theta[0], theta[1], atm.p_bar)
    sig = [xs(sp, atm.nu, T, atm.p_bar, sb=theta[2 + S], wing_cut=atm.wing_cut) for sp in atm.species]
    vmr = np.array([[10.0 ** theta[2 + m]] * len(atm.p_bar) for m in range(S)])
    dt = tau(sig, vmr, atm.p_bar, atm.dp_bar, atm.gravity, atm.mu, atm.kappa_coef)
    return emission(dt, T, atm.nu)


def logl_grad(atm, theta, dobs, sig_obs):
    """(logL, dlogL/dtheta, F0) by forward-mode duals."""
    S = len(atm.species)
    nl = np.array([sp.n for sp in atm.species], dtype=np.int64)
    cat = [_f64(np.concatenate([getattr(sp, f) for sp in atm.species]))
           for f in ("nu_hat", "ln_S0", "elower", "gamma_ref", "n_temp")]
    mass = _f64([sp.mass_amu for sp in atm.species])
    qexp = _f64([sp.q_exponent for sp in atm.species])
    nu, P, dP = _f64(atm.nu), _f64(atm.p_bar), _f64(atm.dp_bar)
    th = _f64(theta)
    d, s = _f64(dobs), _f64(sig_obs)
    grad = np.zeros(3 + S)
    F0 = np.empty(nu.size)
    ll = _load().orc_logl_grad(S, nl.ctypes.data_as(C.POINTER(C.c_int64)), *[_p(v) for v in cat], _p(mass),
                               _p(qexp), nu.size, _p(nu), P.size, _p(P), _p(dP), atm.gravity, atm.mu,
                               atm.kappa_coef, atm.wing_cut, _p(th), _p(d), _p(s), _p(grad), _p(F0))
    return ll, grad, F0


# ------------------------------------------------------------------ MODIT (Sec. 2.1.2)


def modit_fft_length(nu_min, nu_max, N, nu_hat):
    """Smallest power of two M >= 2 (N + farthest centre outside the grid, in
    steps of q = R0 ln nu) + 4: the padded period of the q axis, long enough that
    every line's profile, cut at half a period, covers the whole grid."""
    R0 = (N - 1) / np.log(nu_max / nu_min)
    q = R0 * np.log(np.asarray(nu_hat, dtype=np.float64) / nu_min)
    out = max(0.0, -float(q.min()), float(q.max()) - (N - 1)) if q.size else 0.0
    need = 2 * (N + int(np.ceil(out))) + 4
    return 1 << int(np.ceil(np.log2(need)))


def modit_gamma_grid(gq, n_gamma):
    """n_gamma nodes log-spaced from min to max of the normalised widths gq."""
    lo, hi = np.log(gq.min()), np.log(gq.max())
    if n_gamma < 2 or hi <= lo:
        return np.array([np.exp(lo)] * max(n_gamma, 1))
    return np.exp(lo + (hi - lo) * np.arange(n_gamma) / (n_gamma - 1))


def modit_lsd(lines, nu_min, nu_max, N, T, P_bar, sb, n_gamma, n_fft):
    """Lineshape distribution matrix S_jk of one layer (Sec. 2.1.2): each line
    adds its strength S(T) to the two q nodes around q_l = R0 ln(nu_hat/nu_min)
    and the two log-spaced gamma' nodes around gamma'_l = R0 gamma/nu_hat, with
    weights linear in q and in ln gamma'.  Node q = j is stored at j mod n_fft.
    Returns (lsd [n_gamma][n_fft], gamma' nodes, beta' = R0 beta/nu_hat, R0)."""
    nu_hat = np.asarray(lines.nu_hat, dtype=np.float64)
    R0 = (N - 1) / np.log(nu_max / nu_min)
    S, beta, gam = line_params(lines, T, P_bar, sb)
    q = R0 * np.log(nu_hat / nu_min)
    gq = R0 * gam / nu_hat
    nodes = modit_gamma_grid(gq, n_gamma)
    lsd = np.zeros((n_gamma, n_fft))
    j0 = np.floor(q).astype(np.int64)
    wq = q - j0
    if n_gamma >= 2 and nodes[-1] > nodes[0]:
        t = (np.log(gq) - np.log(nodes[0])) / (np.log(nodes[-1]) - np.log(nodes[0])) * (n_gamma - 1)
        k0 = np.clip(np.floor(t).astype(np.int64), 0, n_gamma - 2)
        wk = t - k0
    else:
        k0 = np.zeros(q.size, dtype=np.int64)
        wk = np.zeros(q.size)
    for dj, fj in ((0, 1.0 - wq), (1, wq)):
        for dk, fk in ((0, 1.0 - wk), (1, wk)):
            kk = np.minimum(k0 + dk, n_gamma - 1)
            np.add.at(lsd, (kk, (j0 + dj) % n_fft), S * fj * fk)
    beta_q = float(np.mean(R0 * beta / nu_hat)) if nu_hat.size else 0.0
    return lsd, nodes, beta_q, R0


def modit_image_sum(M):
    """A(d) = sum over p != 0 of 1/(pi (d + pM)^2) on the period d = -M/2 .. M/2-1
    (index d mod M), from sum_p 1/(d + pM)^2 = (pi/M)^2 / sin^2(pi d/M); near d = 0
    from the Laurent series of csc^2 to avoid cancellation."""
    d = np.arange(M, dtype=np.float64)
    d = np.where(d < M / 2, d, d - M)
    x = np.pi * d / M
    out = np.empty(M)
    small = np.abs(x) < 0.3
    xs = x[small]
    out[small] = (np.pi / M ** 2) * (1.0 / 3 + xs ** 2 / 15 + 2 * xs ** 4 / 189 + xs ** 6 / 675
                                     + 2 * xs ** 8 / 10395)
    xl, dl = x[~small], d[~small]
    out[~small] = ((np.pi / M) ** 2 / np.sin(xl) ** 2 - 1.0 / dl ** 2) / np.pi
    return out


def modit(lines, nu_min, nu_max, N, T, P_bar, sb=1.0, n_gamma=16, n_fft=None):
    """sigma[L][N] on the log grid nu_i = nu_min (nu_max/nu_min)^(i/(N-1)) by
    Eq. MODIT: sigma(q_i) = sum_k IDFT[ DFT(S_.k) K_k(f) ], f the DFT frequency in
    cycles per q step, then sigma(nu) = sigma(q) R0/nu.  K_k is the Voigt
    transform exp(-2 pi^2 beta'^2 f^2 - 2 pi gamma'_k |f|) with the Lorentz
    aliasing removed (reading): the periodic images of each Lorentz profile,
    gamma'_k A(d) to first order in gamma'/M, are subtracted in the transform,
    K_k = exp(-2 pi^2 beta'^2 f^2) (exp(-2 pi gamma'_k |f|) - gamma'_k DFT(A)(f)).
    The result is the linear convolution with each profile cut at half the
    padded period, beyond the grid; there is no other wing cut."""
    T = np.atleast_1d(np.asarray(T, dtype=np.float64))
    P = np.atleast_1d(np.asarray(P_bar, dtype=np.float64))
    if n_fft is None:
        n_fft = modit_fft_length(nu_min, nu_max, N, lines.nu_hat)
    nu = nu_min * (nu_max / nu_min) ** (np.arange(N) / (N - 1))
    f = np.arange(n_fft // 2 + 1) / n_fft
    Ahat = np.fft.rfft(modit_image_sum(n_fft)).real
    out = np.empty((T.size, N))
    for n in range(T.size):
        lsd, nodes, bq, R0 = modit_lsd(lines, nu_min, nu_max, N, T[n], P[n], sb, n_gamma, n_fft)
        gauss = np.exp(-2.0 * np.pi ** 2 * bq ** 2 * f ** 2)
        Y = np.zeros(f.size, dtype=np.complex128)
        for k in range(n_gamma):
            Y += np.fft.rfft(lsd[k]) * gauss * (np.exp(-2.0 * np.pi * nodes[k] * f) - nodes[k] * Ahat)
        y = np.fft.irfft(Y, n=n_fft)
        out[n] = y[:N] * R0 / nu
    return out


# ------------------------------------------------------------------ responses (Sec. 4)

C_KMS = 299792.458  # speed of light in km/s (velocities of Sec. 4 are in km/s)


def rotation_zeta(x, u1, u2):
    """Rigid-rotation kernel of Sec. 4.1: zeta(x) = int I dy / int int I dx dy over the
    unit disk, I = 1 - u1 (1 - mu) - u2 (1 - mu)^2, mu = sqrt(1 - x^2 - y^2),
    written out from that definition with s = sqrt(1 - x^2):
      int I dy = 2s (1 - u1 - u2) + (pi/2) (u1 + 2 u2) s^2 - (4/3) u2 s^3,
      int int I = pi (1 - u1/3 - u2/6).   Zero for |x| >= 1."""
    x = np.asarray(x, dtype=np.float64)
    s = np.sqrt(np.clip(1.0 - x * x, 0.0, None))
    num = 2.0 * s * (1.0 - u1 - u2) + 0.5 * np.pi * (u1 + 2.0 * u2) * s ** 2 - (4.0 / 3.0) * u2 * s ** 3
    return np.where(np.abs(x) < 1.0, num / (np.pi * (1.0 - u1 / 3.0 - u2 / 6.0)), 0.0)


def gauss_ip(v, beta):
    """Gaussian instrumental profile of Sec. 4.2 with standard deviation beta (km/s)."""
    v = np.asarray(v, dtype=np.float64)
    return np.exp(-0.5 * (v / beta) ** 2) / (np.sqrt(2.0 * np.pi) * beta)


def response(F0, nu, nu_out, kernel, rv=0.0):
    """Eq. responsenu: F(nu'_i) = sum_j k(c ln(nu'_i/nu_j) + RV) F0_j / sum_j k(c ln(nu'_i/nu_j)),
    every pair summed (dense)."""
    F0 = np.asarray(F0, dtype=np.float64)
    dv = C_KMS * np.log(np.asarray(nu_out, dtype=np.float64)[:, None] / np.asarray(nu, dtype=np.float64)[None, :])
    return (kernel(dv + rv) @ F0) / kernel(dv).sum(axis=1)


def response_matrix(nu, nu_out, kernel, rv=0.0):
    """The matrix of Eq. responsenu: F = A F0 (its transpose is the adjoint in F0)."""
    dv = C_KMS * np.log(np.asarray(nu_out, dtype=np.float64)[:, None] / np.asarray(nu, dtype=np.float64)[None, :])
    return kernel(dv + rv) / kernel(dv).sum(axis=1)[:, None]


def rotation(F0, nu, vsini, u1, u2):
    """Rotational broadening on the same grid (Sec. 4.1 with Eq. responsenu, RV = 0)."""
    return response(F0, nu, nu, lambda v: rotation_zeta(v / vsini, u1, u2))


def ip_rv(F1, nu, nu_out, beta, rv):
    """Gaussian instrumental profile and radial velocity onto the output grid (Sec. 4.2, Eq. responsenu)."""
    return response(F1, nu, nu_out, lambda v: gauss_ip(v, beta), rv)


# ------------------------------------------------------------------ weak-line pre-filter (App. G)


def contribution_filter(lines, p_bar, dp_bar, T_scan, vmr, g=1e5, mu=2.313, kappa_coef=1e-8, margin=2, sb=1.0,
                        return_psi=False):
    """Lines that can contribute to the emission (App. G).  Per line: the isothermal
    temperature T* of the scan at which S(T) is largest (first on ties); at T*, the
    line-centre layer optical depths dtau_n = (dP_n/g)(vmr/(mu m_u)) S/(sqrt(2 pi) beta)
    erfcx(gamma_n/(sqrt2 beta)) (the optical-depth formula of the model applied to the
    line-centre cross-section); the contribution psi_n = exp(-tau_n) dtau_n P_n/dP_n with
    tau_n = sum_{k<=n} dtau_k; its argmax n_hat (first on ties).  The same for the grey
    continuum (kappa_coef P cm^2/g).  Returns (keep, n_hat per line, n_hat of the
    continuum), keep = n_hat <= n_hat_cont + margin (layer index grows with pressure);
    with return_psi, also psi [L][n] of the lines, to tell which argmax are near-ties."""
    from scipy.special import erfcx
    p = np.asarray(p_bar, dtype=np.float64)
    dp = np.asarray(dp_bar, dtype=np.float64)
    L, n = p.size, lines.nu_hat.size
    best_S = np.full(n, -np.inf)
    best_T = np.zeros(n)
    for T in T_scan:
        S, _, _ = line_params(lines, T, 1.0, sb)
        better = S > best_S
        best_S = np.where(better, S, best_S)
        best_T = np.where(better, T, best_T)
    sig0 = np.empty((L, n))  # line-centre cross-section per layer at each line's T*
    for T in np.unique(best_T):
        idx = np.nonzero(best_T == T)[0]
        sub = lines.subset(idx)
        for k in range(L):
            S, beta, gam = line_params(sub, T, p[k], sb)
            sig0[k, idx] = S / (np.sqrt(2.0 * np.pi) * beta) * erfcx(gam / (np.sqrt(2.0) * beta))
    dtau = tau([sig0], np.full((1, L), vmr), p, dp, g, mu, 0.0)
    dtc = tau([np.zeros((L, 1))], np.zeros((1, L)), p, dp, g, mu, kappa_coef)[:, 0]

    def contribution(dt):
        t = np.cumsum(dt, axis=0)
        return np.exp(-t) * dt * (p / dp).reshape((L,) + (1,) * (dt.ndim - 1))

    psi = contribution(dtau)
    nh = np.argmax(psi, axis=0)
    nc = int(np.argmax(contribution(dtc), axis=0))
    if return_psi:
        return nh <= nc + margin, nh, nc, psi
    return nh <= nc + margin, nh, nc


# ------------------------------------------------------------------ layer temperature prior (Sec. 6.1)


def gp_prior_layers(T, p_bar, T0, a_T=1e6, tau_P=10 ** 0.5, eps=1e-5):
    """The Gaussian-process prior of the layer-by-layer retrieval (Sec. 6.1):
    T ~ N(T0 u, K) with K_ij = a_T k_GP(log10 P_i - log10 P_j; tau_P) + eps a_T delta_ij
    and the RBF kernel k_GP(x; tau) = exp(-x^2 / (2 tau^2)) of Sec. 5.2.3.
    Returns (log p(T), d log p/dT [L], d log p/dT0) from the multivariate normal
    density written out: log p = -r^T K^-1 r / 2 - log det K / 2 - (L/2) log 2 pi,
    r = T - T0 u; d log p/dT = -K^-1 r; d log p/dT0 = u^T K^-1 r.  numpy's solve and
    slogdet are the library steps."""
    T = np.asarray(T, dtype=np.float64)
    lp = np.log10(np.asarray(p_bar, dtype=np.float64))
    L = T.size
    K = a_T * np.exp(-(lp[:, None] - lp[None, :]) ** 2 / (2.0 * tau_P ** 2)) + eps * a_T * np.eye(L)
    r = T - T0
    x = np.linalg.solve(K, r)
    sign, logdet = np.linalg.slogdet(K)
    if sign <= 0:
        return float("nan"), np.full(L, np.nan), float("nan")
    return float(-0.5 * r @ x - 0.5 * logdet - 0.5 * L * np.log(2.0 * np.pi)), -x, float(np.sum(x))
