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
