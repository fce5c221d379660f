"""Thin ctypes binding of libxs (include/xs.h).

Argument marshalling only: every step runs in the CUDA library.  Device memory
comes from PyTorch tensors; the stream is torch's current CUDA stream unless one
is given.  There is no CPU fallback: without the compiled library or a GPU the
calls raise.
"""
from __future__ import annotations

import ctypes as C
import math
import os

import numpy as np
import torch

from . import _build

XS_OK, XS_EINVAL, XS_EUNSORTED, XS_ENOMEM, XS_ECUDA, XS_ETIMEOUT, XS_ETOOBIG = 0, -1, -2, -3, -4, -5, -6
PREC_FP64, PREC_MIXED = 0, 1
MAX_SPECIES = 8

_lib = None


class XsError(RuntimeError):
    def __init__(self, fn, code):
        msg = lib().xs_strerror(code).decode() if _lib is not None else str(code)
        super().__init__(f"{fn} failed: {msg} ({code})")
        self.code = code


class XsLinesC(C.Structure):
    _fields_ = [("n", C.c_int64), ("nu_hat", C.c_void_p), ("ln_S0", C.c_void_p), ("elower", C.c_void_p),
                ("gamma_ref", C.c_void_p), ("n_temp", C.c_void_p), ("mass_amu", C.c_double),
                ("q_exponent", C.c_double)]


class XsModelC(C.Structure):
    _fields_ = [("n_species", C.c_int32), ("species", XsLinesC * MAX_SPECIES), ("nu", C.c_void_p),
                ("N", C.c_int64), ("P_bar", C.c_void_p), ("dP_bar", C.c_void_p), ("L", C.c_int32),
                ("wing_cut", C.c_double), ("gravity", C.c_double), ("mu", C.c_double), ("kappa_coef", C.c_double),
                ("d_obs", C.c_void_p), ("sig_obs", C.c_void_p), ("prec", C.c_int), ("method", C.c_int),
                ("n_gamma", C.c_int32), ("nu_min", C.c_double), ("nu_max", C.c_double),
                ("n_fft", C.c_int64 * MAX_SPECIES), ("cia_alpha", C.c_void_p), ("cia_T", C.c_void_p),
                ("cia_nT", C.c_int32), ("cia_vmr1", C.c_double), ("cia_vmr2", C.c_double)]


def lib():
    """Load libxs.so (building it first if the sources are newer); with the
    environment variable XS_CHECKED=1, the bounds-checked build libxs_checked.so."""
    global _lib
    if _lib is None:
        checked = os.environ.get("XS_CHECKED") == "1"
        path = _build.LIB_CHECKED if checked else _build.LIB
        if not _build.up_to_date(checked):
            path = _build.build(checked=checked)
        if not os.path.exists(path):
            raise RuntimeError("libxs.so is missing; run paper_2105_14782_gb300._build.build()")
        L = C.CDLL(path)
        vp, i64, i32, d, sz, i = C.c_void_p, C.c_int64, C.c_int32, C.c_double, C.c_size_t, C.c_int
        L.xs_strerror.restype = C.c_char_p
        L.xs_strerror.argtypes = [i]
        L.xs_sort_lines_host.argtypes = [i64, vp, vp, vp, vp, vp]
        L.xs_check_sorted.argtypes = [vp, i64, i, vp, vp]
        L.xs_workspace_bytes.restype = sz
        L.xs_workspace_bytes.argtypes = [i64, i64, i32, i]
        L.xs_workspace_min_bytes.restype = sz
        L.xs_workspace_min_bytes.argtypes = [i64, i64, i32, i]
        L.xs_compute.argtypes = [C.POINTER(XsLinesC), vp, i64, vp, vp, i32, d, d, i, vp, vp, sz, vp]
        L.xs_compute_adjoint.argtypes = [C.POINTER(XsLinesC), vp, i64, vp, vp, i32, d, d, i, vp, vp, vp, vp, sz, vp]
        L.tau_layers.argtypes = [C.POINTER(vp), i32, vp, vp, vp, i32, i64, d, d, d, i, vp, vp]
        L.tau_layers_adjoint.argtypes = [C.POINTER(vp), i32, vp, vp, vp, i32, i64, d, d, i, vp, C.POINTER(vp), vp, vp]
        L.emission_spectrum.argtypes = [vp, vp, vp, i32, i64, vp, vp]
        L.emission_workspace_bytes.restype = sz
        L.emission_workspace_bytes.argtypes = [i32, i64]
        L.emission_spectrum_adjoint.argtypes = [vp, vp, vp, vp, i32, i64, vp, vp, vp, sz, vp]
        L.loglike_gauss.argtypes = [vp, vp, vp, i64, vp, vp, vp]
        L.layer_temperatures.argtypes = [d, d, vp, i32, vp, vp]
        L.xs_model_workspace_bytes.restype = sz
        L.xs_model_workspace_bytes.argtypes = [C.POINTER(XsModelC)]
        L.xs_model_forward.argtypes = [C.POINTER(XsModelC), C.POINTER(C.c_double), vp, vp, sz, vp]
        L.xs_model_logl_grad.argtypes = [C.POINTER(XsModelC), C.POINTER(C.c_double), vp, vp, vp, sz, vp]
        L.xs_model_logl_grad_layers.argtypes = [C.POINTER(XsModelC), vp, C.POINTER(C.c_double), d, vp, vp, vp, sz,
                                                vp]
        L.xs_model_forward_keep.argtypes = [C.POINTER(XsModelC), C.POINTER(C.c_double), vp, vp, sz, vp]
        L.xs_model_vjp.argtypes = [C.POINTER(XsModelC), C.POINTER(C.c_double), vp, vp, vp, sz, vp]
        L.xs_profile.argtypes = [i]
        L.xs_profile_read.argtypes = [C.POINTER(C.c_double), C.POINTER(C.c_int64), C.POINTER(C.c_double),
                                      C.POINTER(C.c_int64)]
        L.xs_launch_count.restype = C.c_uint64
        L.xs_check_status.argtypes = [i]
        L.response_rotation.argtypes = [vp, vp, i64, d, d, d, vp, vp]
        L.response_ip_rv.argtypes = [vp, vp, i64, vp, i64, d, d, vp, vp]
        L.response_workspace_bytes.restype = sz
        L.response_workspace_bytes.argtypes = [i64]
        L.response_rotation_adjoint.argtypes = [vp, vp, vp, i64, d, d, d, vp, vp, vp, sz, vp]
        L.response_ip_rv_adjoint.argtypes = [vp, vp, vp, i64, vp, i64, d, d, vp, vp, vp, sz, vp]
        L.tau_cia.argtypes = [vp, vp, i32, vp, vp, vp, i32, i64, d, d, d, d, i, vp, vp]
        L.tau_cia_adjoint.argtypes = [vp, vp, vp, i32, vp, vp, vp, i32, i64, d, d, d, d, vp, vp]
        L.lines_contribution_filter.argtypes = [C.POINTER(XsLinesC), vp, vp, i32, C.POINTER(C.c_double), i32, d, d, d,
                                                d, d, i32, vp, vp, vp]
        L.modit_adjoint_workspace_bytes.restype = sz
        L.modit_adjoint_workspace_bytes.argtypes = [i64, i32, i32, i64, i]
        L.modit_compute_adjoint.argtypes = [C.POINTER(XsLinesC), d, d, i64, vp, vp, i32, d, i32, i64, i, vp, vp, vp,
                                            vp, sz, vp]
        L.modit_workspace_bytes.restype = sz
        L.modit_workspace_bytes.argtypes = [i64, i32, i32, i64, i]
        L.modit_compute.argtypes = [C.POINTER(XsLinesC), d, d, i64, vp, vp, i32, d, i32, i64, i, vp, vp, sz, vp]
        L.gp_prior_workspace_bytes.restype = sz
        L.gp_prior_workspace_bytes.argtypes = [i32]
        L.gp_prior_layers.argtypes = [vp, vp, i32, d, d, d, d, vp, vp, sz, vp]
        _lib = L
    return _lib


def _check(fn, code):
    if code != XS_OK:
        raise XsError(fn, code)


def _stream(stream):
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def _dev(t):
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.is_contiguous()):
        raise ValueError("expected a contiguous CUDA tensor")
    return C.c_void_p(t.data_ptr())


def _ws(nbytes, device):
    return torch.empty(max(int(nbytes), 256), dtype=torch.uint8, device=device)


class DeviceLines:
    """A line list sorted by centre (libxs's host sort) and resident on the GPU."""

    def __init__(self, lines, device="cuda"):
        arrs = [np.array(a, dtype=np.float64, copy=True) for a in lines.arrays()]
        n = arrs[0].size
        _check("xs_sort_lines_host", lib().xs_sort_lines_host(n, *[a.ctypes.data_as(C.c_void_p) for a in arrs]))
        self.n = n
        self.mass_amu = float(lines.mass_amu)
        self.q_exponent = float(lines.q_exponent)
        self.tensors = [torch.from_numpy(a).to(device) for a in arrs]
        self.nu_hat, self.ln_S0, self.elower, self.gamma_ref, self.n_temp = self.tensors

    def select(self, mask):
        """The lines where mask (bool device tensor [n]) is true, same order, on the device."""
        out = DeviceLines.__new__(DeviceLines)
        out.tensors = [t[mask].contiguous() for t in self.tensors]
        out.n = out.tensors[0].numel()
        out.mass_amu, out.q_exponent = self.mass_amu, self.q_exponent
        out.nu_hat, out.ln_S0, out.elower, out.gamma_ref, out.n_temp = out.tensors
        return out

    def struct(self):
        ptr = [t.data_ptr() if self.n else None for t in self.tensors]
        return XsLinesC(self.n, *ptr, self.mass_amu, self.q_exponent)


def check_sorted(v, strict=False, stream=None):
    flag = torch.zeros(1, dtype=torch.int32, device=v.device)
    return lib().xs_check_sorted(_dev(v), v.numel(), int(strict), _dev(flag), _stream(stream))


def workspace_bytes(n_lines, N, L, prec):
    return lib().xs_workspace_bytes(n_lines, N, L, prec)


def xs_compute(lines: DeviceLines, nu, T, P_bar, broad_scale=1.0, wing_cut=25.0, prec=PREC_MIXED, out=None,
               workspace=None, stream=None):
    N, L = nu.numel(), T.numel()
    dt = torch.float32 if prec == PREC_MIXED else torch.float64
    if out is None:
        out = torch.empty((L, N), dtype=dt, device=nu.device)
    if workspace is None:
        workspace = _ws(workspace_bytes(lines.n, N, L, prec), nu.device)
    s = lines.struct()
    _check("xs_compute", lib().xs_compute(C.byref(s), _dev(nu), N, _dev(T), _dev(P_bar), L, float(broad_scale),
                                          float(wing_cut), prec, _dev(out), _dev(workspace), workspace.numel(),
                                          _stream(stream)))
    return out


def xs_compute_adjoint(lines: DeviceLines, nu, T, P_bar, g_sigma, broad_scale=1.0, wing_cut=25.0, prec=PREC_MIXED,
                       workspace=None, stream=None):
    N, L = nu.numel(), T.numel()
    g_T = torch.empty(L, dtype=torch.float64, device=nu.device)
    g_b = torch.empty(1, dtype=torch.float64, device=nu.device)
    if workspace is None:
        workspace = _ws(workspace_bytes(lines.n, N, L, prec), nu.device)
    s = lines.struct()
    _check("xs_compute_adjoint", lib().xs_compute_adjoint(
        C.byref(s), _dev(nu), N, _dev(T), _dev(P_bar), L, float(broad_scale), float(wing_cut), prec, _dev(g_sigma),
        _dev(g_T), _dev(g_b), _dev(workspace), workspace.numel(), _stream(stream)))
    return g_T, g_b


def modit_fft_length(nu_min, nu_max, N, lines: "DeviceLines", span=None):
    """Smallest power of two >= 2 (N + farthest centre outside the grid, in q
    steps) + 4, so that every profile covers the whole grid.  span = (lowest,
    highest centre), when given, replaces the read of the device list."""
    R0 = (N - 1) / math.log(nu_max / nu_min)
    if span is not None or lines.n:
        lo, hi = span if span is not None else (float(lines.nu_hat[0].item()), float(lines.nu_hat[-1].item()))
        out = max(0.0, -R0 * math.log(lo / nu_min), R0 * math.log(hi / nu_min) - (N - 1))
    else:
        out = 0.0
    need = 2 * (N + int(math.ceil(out))) + 4
    return 1 << int(math.ceil(math.log2(need)))


def modit_compute(lines: DeviceLines, nu_min, nu_max, N, T, P_bar, broad_scale=1.0, n_gamma=16, n_fft=None,
                  prec=PREC_FP64, out=None, workspace=None, stream=None):
    """MODIT cross-section sigma[L][N] on the log grid nu_min .. nu_max (N points)."""
    L = T.numel()
    if n_fft is None:
        n_fft = modit_fft_length(nu_min, nu_max, N, lines)
    dt = torch.float32 if prec == PREC_MIXED else torch.float64
    if out is None:
        out = torch.empty((L, N), dtype=dt, device=T.device)
    if workspace is None:
        workspace = _ws(lib().modit_workspace_bytes(lines.n, L, n_gamma, n_fft, prec), T.device)
    s = lines.struct()
    _check("modit_compute", lib().modit_compute(C.byref(s), float(nu_min), float(nu_max), N, _dev(T), _dev(P_bar), L,
                                                float(broad_scale), n_gamma, n_fft, prec, _dev(out),
                                                _dev(workspace), workspace.numel(), _stream(stream)))
    return out


def response_rotation(F0, nu, vsini, u1=0.0, u2=0.0, out=None, stream=None):
    """Rigid-rotation broadening (Sec. 4.1) of F0 on its own grid nu (km/s)."""
    out = torch.empty_like(F0) if out is None else out
    _check("response_rotation", lib().response_rotation(_dev(F0), _dev(nu), nu.numel(), float(vsini), float(u1),
                                                        float(u2), _dev(out), _stream(stream)))
    return out


def response_ip_rv(F1, nu, nu_out, beta, rv=0.0, out=None, stream=None):
    """Gaussian instrumental profile (std beta, km/s) and radial velocity rv onto nu_out (Sec. 4.2)."""
    out = torch.empty(nu_out.numel(), dtype=torch.float64, device=F1.device) if out is None else out
    _check("response_ip_rv", lib().response_ip_rv(_dev(F1), _dev(nu), nu.numel(), _dev(nu_out), nu_out.numel(),
                                                  float(beta), float(rv), _dev(out), _stream(stream)))
    return out


def response_rotation_adjoint(g_F1, F0, nu, vsini, u1=0.0, u2=0.0, stream=None):
    g_F0 = torch.empty_like(F0)
    g_v = torch.empty(1, dtype=torch.float64, device=F0.device)
    ws = _ws(lib().response_workspace_bytes(nu.numel()), F0.device)
    _check("response_rotation_adjoint", lib().response_rotation_adjoint(
        _dev(g_F1), _dev(F0), _dev(nu), nu.numel(), float(vsini), float(u1), float(u2), _dev(g_F0), _dev(g_v),
        _dev(ws), ws.numel(), _stream(stream)))
    return g_F0, g_v


def response_ip_rv_adjoint(g_F, F1, nu, nu_out, beta, rv=0.0, stream=None):
    g_F1 = torch.empty_like(F1)
    g_rv = torch.empty(1, dtype=torch.float64, device=F1.device)
    ws = _ws(lib().response_workspace_bytes(nu_out.numel()), F1.device)
    _check("response_ip_rv_adjoint", lib().response_ip_rv_adjoint(
        _dev(g_F), _dev(F1), _dev(nu), nu.numel(), _dev(nu_out), nu_out.numel(), float(beta), float(rv), _dev(g_F1),
        _dev(g_rv), _dev(ws), ws.numel(), _stream(stream)))
    return g_F1, g_rv


def tau_cia(alpha, T_grid, T, P_bar, dP_bar, vmr1, vmr2, gravity=1e5, mu=2.313, out=None, stream=None):
    """Collision-induced absorption optical depth [L][N] (Sec. 2.4); added to out when given."""
    L, N = T.numel(), alpha.shape[1]
    acc = out is not None
    out = torch.empty((L, N), dtype=torch.float64, device=T.device) if out is None else out
    _check("tau_cia", lib().tau_cia(_dev(alpha), _dev(T_grid), T_grid.numel(), _dev(T), _dev(P_bar), _dev(dP_bar), L,
                                    N, float(vmr1), float(vmr2), float(gravity), float(mu), int(acc), _dev(out),
                                    _stream(stream)))
    return out


def tau_cia_adjoint(g_dtau, alpha, T_grid, T, P_bar, dP_bar, vmr1, vmr2, gravity=1e5, mu=2.313, stream=None):
    g_T = torch.zeros(T.numel(), dtype=torch.float64, device=T.device)
    _check("tau_cia_adjoint", lib().tau_cia_adjoint(
        _dev(g_dtau), _dev(alpha), _dev(T_grid), T_grid.numel(), _dev(T), _dev(P_bar), _dev(dP_bar), T.numel(),
        alpha.shape[1], float(vmr1), float(vmr2), float(gravity), float(mu), _dev(g_T), _stream(stream)))
    return g_T


def contribution_filter(lines: DeviceLines, P_bar, dP_bar, T_scan, vmr, gravity=1e5, mu=2.313, kappa_coef=1e-8,
                        broad_scale=1.0, margin=2, stream=None):
    """Weak-line pre-filter of App. G: (keep bool [n], n_hat int32 [n]) on the device."""
    keep = torch.zeros(max(lines.n, 1), dtype=torch.uint8, device=P_bar.device)
    nh = torch.zeros(max(lines.n, 1), dtype=torch.int32, device=P_bar.device)
    ts = (C.c_double * len(T_scan))(*[float(t) for t in T_scan])
    s = lines.struct()
    _check("lines_contribution_filter", lib().lines_contribution_filter(
        C.byref(s), _dev(P_bar), _dev(dP_bar), P_bar.numel(), ts, len(T_scan), float(vmr), float(gravity), float(mu),
        float(kappa_coef), float(broad_scale), int(margin), _dev(keep), _dev(nh), _stream(stream)))
    return keep[:lines.n].bool(), nh[:lines.n]


def modit_compute_adjoint(lines: DeviceLines, nu_min, nu_max, N, T, P_bar, g_sigma, broad_scale=1.0, n_gamma=16,
                          n_fft=None, prec=PREC_FP64, workspace=None, stream=None):
    """(g_T [L], g_broad [1]) of sum(g_sigma * modit_compute(...))."""
    L = T.numel()
    if n_fft is None:
        n_fft = modit_fft_length(nu_min, nu_max, N, lines)
    g_T = torch.empty(L, dtype=torch.float64, device=T.device)
    g_b = torch.empty(1, dtype=torch.float64, device=T.device)
    if workspace is None:
        workspace = _ws(lib().modit_adjoint_workspace_bytes(lines.n, L, n_gamma, n_fft, prec), T.device)
    s = lines.struct()
    _check("modit_compute_adjoint", lib().modit_compute_adjoint(
        C.byref(s), float(nu_min), float(nu_max), N, _dev(T), _dev(P_bar), L, float(broad_scale), n_gamma, n_fft,
        prec, _dev(g_sigma), _dev(g_T), _dev(g_b), _dev(workspace), workspace.numel(), _stream(stream)))
    return g_T, g_b


def _ptrs(ts):
    arr = (C.c_void_p * len(ts))(*[t.data_ptr() if t is not None else None for t in ts])
    return arr


def tau_layers(sigmas, vmr, P_bar, dP_bar, gravity=1e5, mu=2.313, kappa_coef=1e-8, prec=PREC_MIXED, stream=None):
    L, N = sigmas[0].shape
    dtau = torch.empty((L, N), dtype=torch.float64, device=P_bar.device)
    _check("tau_layers", lib().tau_layers(_ptrs(sigmas), len(sigmas), _dev(vmr), _dev(P_bar), _dev(dP_bar), L, N,
                                          float(gravity), float(mu), float(kappa_coef), prec, _dev(dtau),
                                          _stream(stream)))
    return dtau


def tau_layers_adjoint(sigmas, vmr, P_bar, dP_bar, g_dtau, gravity=1e5, mu=2.313, prec=PREC_MIXED, stream=None):
    L, N = sigmas[0].shape
    gs = [torch.empty((L, N), dtype=torch.float64, device=P_bar.device) for _ in sigmas]
    gv = torch.empty((len(sigmas), L), dtype=torch.float64, device=P_bar.device)
    _check("tau_layers_adjoint", lib().tau_layers_adjoint(
        _ptrs(sigmas), len(sigmas), _dev(vmr), _dev(P_bar), _dev(dP_bar), L, N, float(gravity), float(mu), prec,
        _dev(g_dtau), _ptrs(gs), _dev(gv), _stream(stream)))
    return gs, gv


def emission_spectrum(dtau, T, nu, stream=None):
    L, N = dtau.shape
    F0 = torch.empty(N, dtype=torch.float64, device=dtau.device)
    _check("emission_spectrum", lib().emission_spectrum(_dev(dtau), _dev(T), _dev(nu), L, N, _dev(F0),
                                                        _stream(stream)))
    return F0


def emission_spectrum_adjoint(g_F0, dtau, T, nu, stream=None):
    L, N = dtau.shape
    g_dtau = torch.empty_like(dtau)
    g_T = torch.empty(L, dtype=torch.float64, device=dtau.device)
    ws = _ws(lib().emission_workspace_bytes(L, N), dtau.device)
    _check("emission_spectrum_adjoint", lib().emission_spectrum_adjoint(
        _dev(g_F0), _dev(dtau), _dev(T), _dev(nu), L, N, _dev(g_dtau), _dev(g_T), _dev(ws), ws.numel(),
        _stream(stream)))
    return g_dtau, g_T


def loglike_gauss(F, d, s, stream=None):
    out = torch.empty(1, dtype=torch.float64, device=F.device)
    gF = torch.empty_like(F)
    _check("loglike_gauss", lib().loglike_gauss(_dev(F), _dev(d), _dev(s), F.numel(), _dev(out), _dev(gF),
                                                _stream(stream)))
    return out, gF


def layer_temperatures(T0, alpha, P_bar, stream=None):
    T = torch.empty_like(P_bar)
    _check("layer_temperatures", lib().layer_temperatures(float(T0), float(alpha), _dev(P_bar), P_bar.numel(),
                                                          _dev(T), _stream(stream)))
    return T


def gp_prior_layers(T, P_bar, T0, a_T=1e6, tau_P=10 ** 0.5, eps=1e-5, stream=None):
    """Gaussian-process prior of the layer temperatures (Sec. 6.1): device tensor
    [log p(T), d log p/dT_0 .. d log p/dT_{L-1}, d log p/dT0]."""
    L = T.numel()
    out = torch.empty(L + 2, dtype=torch.float64, device=T.device)
    ws = _ws(lib().gp_prior_workspace_bytes(L), T.device)
    _check("gp_prior_layers", lib().gp_prior_layers(_dev(T), _dev(P_bar), L, float(T0), float(a_T), float(tau_P),
                                                    float(eps), _dev(out), _dev(ws), ws.numel(), _stream(stream)))
    return out


def profile(enable: bool):
    """Start (True) or stop (False) event timing of the line-sum kernels."""
    _check("xs_profile", lib().xs_profile(int(enable)))


def profile_read():
    """(forward ms, forward launches, adjoint ms, adjoint launches) since profile(True)."""
    a, b, c, d = C.c_double(), C.c_int64(), C.c_double(), C.c_int64()
    _check("xs_profile_read", lib().xs_profile_read(C.byref(a), C.byref(b), C.byref(c), C.byref(d)))
    return a.value, b.value, c.value, d.value


def check_status(clear=True) -> int:
    """0 unless a bounds check of the checked build failed (file * 100000 + line)."""
    return int(lib().xs_check_status(int(clear)))


def launch_count() -> int:
    return int(lib().xs_launch_count())


class EmissionModel:
    """Species line lists, grid, layers and (optionally) an observed spectrum,
    resident on one GPU, with the composite forward and log-likelihood-gradient
    calls of libxs.  theta = (T0, alpha, log10 vmr_0..log10 vmr_{S-1}, s_b)."""

    def __init__(self, atm, prec=PREC_MIXED, device="cuda", d_obs=None, sig_obs=None, lines=None, method="lpf",
                 n_gamma=16, cia=None):
        """cia: optional (T_grid [nT], alpha [nT][N], vmr1, vmr2), a collision-induced
        absorption pair added to the optical depth (Sec. 2.4)."""
        self.device = torch.device(device)
        self.cia = None
        if cia is not None:
            Tg, alpha, v1, v2 = cia
            f64_ = dict(dtype=torch.float64, device=self.device)
            self.cia = (torch.as_tensor(np.asarray(Tg), **f64_).contiguous(),
                        torch.as_tensor(np.asarray(alpha), **f64_).contiguous(), float(v1), float(v2))
        self.prec = prec
        self.method, self.n_gamma = method, int(n_gamma)
        if method == "modit":
            nu = np.asarray(atm.nu, dtype=np.float64)
            want = nu[0] * (nu[-1] / nu[0]) ** (np.arange(nu.size) / (nu.size - 1))
            if not np.allclose(nu, want, rtol=1e-13, atol=0):
                raise ValueError("MODIT needs the log grid nu_min (nu_max/nu_min)^(i/(N-1))")
        elif method != "lpf":
            raise ValueError(f"unknown cross-section method {method!r}")
        self.species = lines if lines is not None else [DeviceLines(sp, device) for sp in atm.species]
        f64 = dict(dtype=torch.float64, device=self.device)
        self.nu = torch.as_tensor(np.asarray(atm.nu), **f64)
        self.P = torch.as_tensor(np.asarray(atm.p_bar), **f64)
        self.dP = torch.as_tensor(np.asarray(atm.dp_bar), **f64)
        self.atm = atm
        self.S = len(self.species)
        self.N, self.L = self.nu.numel(), self.P.numel()
        self.d_obs = None if d_obs is None else torch.as_tensor(np.asarray(d_obs), **f64)
        self.sig_obs = None if sig_obs is None else torch.as_tensor(np.asarray(sig_obs), **f64)
        self._c = self._struct()
        self.ws = _ws(lib().xs_model_workspace_bytes(C.byref(self._c)), self.device)
        self.out = torch.empty(1 + 3 + self.S, **f64)
        self.F0 = torch.empty(self.N, **f64)

    def _struct(self):
        sp = (XsLinesC * MAX_SPECIES)()
        for i, s in enumerate(self.species):
            sp[i] = s.struct()
        c = self._struct_base(sp)
        if self.method == "modit":
            nu0, nu1 = float(self.atm.nu[0]), float(self.atm.nu[-1])
            c.method, c.n_gamma, c.nu_min, c.nu_max = 1, self.n_gamma, nu0, nu1
            for i, sp_ in enumerate(self.species):
                c.n_fft[i] = modit_fft_length(nu0, nu1, self.N, sp_)
        if self.cia is not None:
            Tg, alpha, v1, v2 = self.cia
            c.cia_alpha, c.cia_T, c.cia_nT, c.cia_vmr1, c.cia_vmr2 = alpha.data_ptr(), Tg.data_ptr(), Tg.numel(), v1, v2
        return c

    def _struct_base(self, sp):
        a = self.atm
        return XsModelC(self.S, sp, self.nu.data_ptr(), self.N, self.P.data_ptr(), self.dP.data_ptr(), self.L,
                        float(a.wing_cut), float(a.gravity), float(a.mu), float(a.kappa_coef),
                        None if self.d_obs is None else self.d_obs.data_ptr(),
                        None if self.sig_obs is None else self.sig_obs.data_ptr(), self.prec)

    def set_observation(self, d_obs, sig_obs):
        f64 = dict(dtype=torch.float64, device=self.device)
        self.d_obs = torch.as_tensor(d_obs, **f64).contiguous()
        self.sig_obs = torch.as_tensor(sig_obs, **f64).contiguous()
        self._c = self._struct()

    def forward(self, theta, out=None, stream=None):
        th = (C.c_double * len(theta))(*[float(v) for v in theta])
        F0 = self.F0 if out is None else out
        _check("xs_model_forward", lib().xs_model_forward(C.byref(self._c), th, _dev(F0), _dev(self.ws),
                                                          self.ws.numel(), _stream(stream)))
        return F0

    def logl_grad_async(self, theta, out=None, F0=None, stream=None):
        """Launches the forward + adjoint; returns the device tensor
        [logL, dlogL/dtheta...] (valid once the stream reaches this point)."""
        th = (C.c_double * len(theta))(*[float(v) for v in theta])
        o = self.out if out is None else out
        _check("xs_model_logl_grad", lib().xs_model_logl_grad(
            C.byref(self._c), th, _dev(o), None if F0 is None else _dev(F0), _dev(self.ws), self.ws.numel(),
            _stream(stream)))
        return o

    def logl_grad(self, theta, stream=None):
        o = self.logl_grad_async(theta, stream=stream).cpu().numpy()
        return float(o[0]), o[1:].copy()


    def logl_grad_layers(self, T, log10_vmr, broad_scale=1.0, stream=None):
        """logL and its gradient in the per-layer temperatures T [L] (device tensor),
        the log10 mixing ratios and the broadening scale: (logL, g_T [L], g_vmr [S], g_b)."""
        lv = (C.c_double * self.S)(*[float(v) for v in log10_vmr])
        o = torch.empty(2 + self.L + self.S, dtype=torch.float64, device=self.device)
        T = torch.as_tensor(T, dtype=torch.float64, device=self.device).contiguous()
        _check("xs_model_logl_grad_layers", lib().xs_model_logl_grad_layers(
            C.byref(self._c), _dev(T), lv, float(broad_scale), _dev(o), None, _dev(self.ws), self.ws.numel(),
            _stream(stream)))
        o = o.cpu().numpy()
        return float(o[0]), o[1:1 + self.L], o[1 + self.L:1 + self.L + self.S], float(o[1 + self.L + self.S])

    def forward_keep(self, theta, out=None, stream=None):
        """F0 at theta, keeping the reverse sweep's state in the workspace (for vjp)."""
        th = (C.c_double * len(theta))(*[float(v) for v in theta])
        F0 = self.F0 if out is None else out
        _check("xs_model_forward_keep", lib().xs_model_forward_keep(C.byref(self._c), th, _dev(F0), _dev(self.ws),
                                                                    self.ws.numel(), _stream(stream)))
        return F0

    def vjp(self, theta, g_F0, stream=None):
        """g_F0 . dF0/dtheta after forward_keep(theta): device tensor [3 + S]."""
        th = (C.c_double * len(theta))(*[float(v) for v in theta])
        _check("xs_model_vjp", lib().xs_model_vjp(C.byref(self._c), th, _dev(g_F0), _dev(self.out), _dev(self.ws),
                                                  self.ws.numel(), _stream(stream)))
        return self.out[1:]


class ObservedModel:
    """The model of Sec. 5's fit: emission F0 on the model grid, rigid rotation
    (vsini, limb darkening u1, u2), Gaussian IP (beta) with radial velocity onto the
    observed grid, Gaussian likelihood there (Eq. likelihood).  Parameters
    theta = (T0, alpha, log10 vmr_0..log10 vmr_{S-1}, s_b, vsini, RV); the gradient
    comes from the responses' adjoints and the composite model's vector-Jacobian
    product."""

    def __init__(self, model: EmissionModel, nu_obs, d_obs, sig_obs, beta, u1=0.0, u2=0.0):
        f64 = dict(dtype=torch.float64, device=model.device)
        self.m = model
        self.nu_obs = torch.as_tensor(np.asarray(nu_obs), **f64)
        self.d = torch.as_tensor(np.asarray(d_obs), **f64)
        self.s = torch.as_tensor(np.asarray(sig_obs), **f64)
        self.beta, self.u1, self.u2 = float(beta), float(u1), float(u2)
        self.out = torch.empty(2, **f64)

    def spectrum(self, theta, keep=False):
        th, vsini, rv = list(theta[:-2]), float(theta[-2]), float(theta[-1])
        F0 = self.m.forward_keep(th) if keep else self.m.forward(th)
        F1 = response_rotation(F0, self.m.nu, vsini, self.u1, self.u2)
        return F0, F1, response_ip_rv(F1, self.m.nu, self.nu_obs, self.beta, rv)

    def logl_grad(self, theta):
        th, vsini, rv = list(theta[:-2]), float(theta[-2]), float(theta[-1])
        F0, F1, F = self.spectrum(theta, keep=True)
        ll, gF = loglike_gauss(F, self.d, self.s)
        gF1, g_rv = response_ip_rv_adjoint(gF, F1, self.m.nu, self.nu_obs, self.beta, rv)
        gF0, g_vsini = response_rotation_adjoint(gF1, F0, self.m.nu, vsini, self.u1, self.u2)
        g = self.m.vjp(th, gF0)
        grad = torch.cat([g, g_vsini, g_rv]).cpu().numpy()
        return float(ll.item()), grad


class SpectrumLogL(torch.autograd.Function):
    """logL(theta) with the gradient from libxs's hand-written adjoint kernels."""

    @staticmethod
    def forward(ctx, theta, model):
        th = theta.detach().cpu().double().tolist()
        o = model.logl_grad_async(th).clone()
        ctx.save_for_backward(o[1:].to(theta.device, theta.dtype))
        return o[0:1].to(theta.device, theta.dtype).reshape(())

    @staticmethod
    def backward(ctx, g):
        (grad,) = ctx.saved_tensors
        return g * grad, None


def log_likelihood(theta, model):
    return SpectrumLogL.apply(theta, model)


LN10 = math.log(10.0)
