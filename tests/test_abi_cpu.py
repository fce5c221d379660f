"""Host-side checks of libxs that need no GPU: every function declared in
include/xs.h is exported, and the pure host logic (sort, workspace sizing,
status strings, argument rejection before any launch) behaves."""
import ctypes as C
import os
import re

import numpy as np
import pytest

import workloads as W
from paper_2105_14782_gb300 import _build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    txt = open(os.path.join(ROOT, "include", "xs.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(\w+)\s*\(", txt, flags=re.M)
    return sorted(set(n for n in names if n not in ("if", "return")))


@pytest.fixture(scope="module")
def lib():
    path = _build.build()
    return C.CDLL(path)


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert len(names) >= 17
    for n in names:
        assert hasattr(lib, n), n


def test_host_sort_is_stable_and_carries_fields(lib):
    ln = W.water_like(5000, seed=9)
    nu = ln.nu_hat.copy()
    nu[10] = nu[20]  # a tie
    arrs = [nu, ln.ln_S0.copy(), ln.elower.copy(), ln.gamma_ref.copy(), ln.n_temp.copy()]
    ref = np.argsort(nu, kind="stable")
    want = [a[ref] for a in arrs]
    lib.xs_sort_lines_host.argtypes = [C.c_int64] + [C.c_void_p] * 5
    assert lib.xs_sort_lines_host(nu.size, *[a.ctypes.data_as(C.c_void_p) for a in arrs]) == 0
    for a, b in zip(arrs, want):
        assert np.array_equal(a, b)


def test_workspace_sizes_and_strings(lib):
    lib.xs_workspace_bytes.restype = C.c_size_t
    lib.xs_workspace_bytes.argtypes = [C.c_int64, C.c_int64, C.c_int32, C.c_int]
    lib.xs_workspace_min_bytes.restype = C.c_size_t
    lib.xs_workspace_min_bytes.argtypes = [C.c_int64, C.c_int64, C.c_int32, C.c_int]
    full = lib.xs_workspace_bytes(220_000, 20_000, 100, 1)
    small = lib.xs_workspace_min_bytes(220_000, 20_000, 100, 1)
    assert full > small > 0
    assert lib.xs_workspace_bytes(220_000, 20_000, 100, 0) > full  # FP64 records are twice as wide
    assert lib.xs_workspace_bytes(10, 0, 1, 1) == 0
    lib.xs_strerror.restype = C.c_char_p
    assert lib.xs_strerror(-2).decode().startswith("line centres")


def test_invalid_arguments_rejected_before_launch(lib):
    lib.xs_compute.argtypes = [C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p, C.c_int32, C.c_double,
                               C.c_double, C.c_int, C.c_void_p, C.c_void_p, C.c_size_t, C.c_void_p]
    assert lib.xs_compute(None, None, 10, None, None, 1, 1.0, 25.0, 1, None, None, 0, None) == -1
    lib.emission_spectrum.argtypes = [C.c_void_p] * 3 + [C.c_int32, C.c_int64, C.c_void_p, C.c_void_p]
    assert lib.emission_spectrum(None, None, None, 0, 5, None, None) == -1
    lib.layer_temperatures.argtypes = [C.c_double, C.c_double, C.c_void_p, C.c_int32, C.c_void_p, C.c_void_p]
    assert lib.layer_temperatures(-5.0, 0.1, None, 3, None, None) == -1


def test_workspace_queries_of_the_other_entry_points(lib):
    lib.modit_workspace_bytes.restype = C.c_size_t
    lib.modit_workspace_bytes.argtypes = [C.c_int64, C.c_int32, C.c_int32, C.c_int64, C.c_int]
    lib.modit_adjoint_workspace_bytes.restype = C.c_size_t
    lib.modit_adjoint_workspace_bytes.argtypes = lib.modit_workspace_bytes.argtypes
    a = lib.modit_workspace_bytes(200_000, 100, 16, 65536, 0)
    b = lib.modit_workspace_bytes(200_000, 100, 16, 65536, 1)
    assert a > b > 0  # FP32 distribution and transforms take less
    # distribution + transform + output rows at least
    assert a >= 100 * 16 * 65536 * 8 + 100 * 16 * 32769 * 16
    assert lib.modit_adjoint_workspace_bytes(200_000, 100, 16, 65536, 0) > a
    assert lib.modit_workspace_bytes(10, 1, 16, 1000, 0) == 0   # not a power of two
    assert lib.modit_workspace_bytes(10, 1, 33, 1024, 0) == 0   # too many gamma nodes
    assert lib.modit_workspace_bytes(10, 0, 16, 1024, 0) == 0   # no layers
    lib.response_workspace_bytes.restype = C.c_size_t
    lib.response_workspace_bytes.argtypes = [C.c_int64]
    assert lib.response_workspace_bytes(0) == 0
    assert lib.response_workspace_bytes(1000) >= 1000 * 8


def test_new_entry_points_reject_bad_arguments_before_launch(lib):
    vp = C.c_void_p
    lib.modit_compute.argtypes = [vp, C.c_double, C.c_double, C.c_int64, vp, vp, C.c_int32, C.c_double, C.c_int32,
                                  C.c_int64, C.c_int, vp, vp, C.c_size_t, vp]
    assert lib.modit_compute(None, 4340.0, 4390.0, 100, None, None, 1, 1.0, 16, 256, 0, None, None, 0, None) == -1
    lib.response_rotation.argtypes = [vp, vp, C.c_int64, C.c_double, C.c_double, C.c_double, vp, vp]
    assert lib.response_rotation(None, None, 10, 30.0, 0.4, 0.2, None, None) == -1
    lib.response_ip_rv.argtypes = [vp, vp, C.c_int64, vp, C.c_int64, C.c_double, C.c_double, vp, vp]
    assert lib.response_ip_rv(None, None, 10, None, 10, 2.0, 0.0, None, None) == -1
    lib.lines_contribution_filter.argtypes = [vp, vp, vp, C.c_int32, vp, C.c_int32, C.c_double, C.c_double,
                                              C.c_double, C.c_double, C.c_double, C.c_int32, vp, vp, vp]
    assert lib.lines_contribution_filter(None, None, None, 10, None, 1, 1e-3, 1e5, 2.313, 0.1, 1.0, 2, None, None,
                                         None) == -1
    lib.xs_model_vjp.argtypes = [vp] * 7
    assert lib.xs_model_vjp(None, None, None, None, None, None, None) == -1
    lib.xs_model_forward_keep.argtypes = [vp] * 6
    assert lib.xs_model_forward_keep(None, None, None, None, None, None) == -1
    lib.xs_model_logl_grad_layers.argtypes = [vp, vp, vp, C.c_double, vp, vp, vp, C.c_size_t, vp]
    assert lib.xs_model_logl_grad_layers(None, None, None, 1.0, None, None, None, 0, None) == -1


def test_gp_prior_rejects_bad_arguments(lib):
    lib.gp_prior_workspace_bytes.restype = C.c_size_t
    lib.gp_prior_workspace_bytes.argtypes = [C.c_int32]
    assert lib.gp_prior_workspace_bytes(100) == 8 * (100 * 100 + 100)
    assert lib.gp_prior_workspace_bytes(0) == 0
    assert lib.gp_prior_workspace_bytes(1025) == 0
    vp, d = C.c_void_p, C.c_double
    lib.gp_prior_layers.argtypes = [vp, vp, C.c_int32, d, d, d, d, vp, vp, C.c_size_t, vp]
    buf = (C.c_double * 16)()
    p = C.cast(buf, vp)
    ok = (p, p, 2, 1300.0, 1e6, 3.0, 1e-5, p, p, 8 * 6)
    for k, bad in ((0, None), (2, 0), (2, 1025), (3, float("nan")), (4, 0.0), (5, -1.0), (6, -1e-5), (9, 8 * 5)):
        args = list(ok)
        args[k] = bad
        assert lib.gp_prior_layers(*args, None) == -1, (k, bad)


def test_bounds_checked_build_is_marked(lib):
    """The normal library reports no checked build and a clean status without a
    GPU call path; the checked variant (-DXS_CHECKED) reports itself."""
    lib.xs_checked_build.restype = C.c_int
    assert lib.xs_checked_build() == 0
    checked = C.CDLL(_build.build(checked=True))
    checked.xs_checked_build.restype = C.c_int
    assert checked.xs_checked_build() == 1
    for n in _declared():
        assert hasattr(checked, n), n
