"""xs_compute_noalloc: the cross-section entry point for callers that cannot
allocate device memory (host callbacks and real-time loops that must not block
in the allocator, plugins whose host process owns the memory pool).  Its scratch
is a fixed array inside libxs, so it must give the same cross-section as
xs_compute with a caller workspace, call after call.  This file is collected
last on purpose."""
import ctypes as C

import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def xs():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_2105_14782_gb300 import xs as _xs
    L = _xs.lib()
    L.xs_compute_noalloc.argtypes = [C.POINTER(_xs.XsLinesC), C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p,
                                     C.c_int32, C.c_double, C.c_double, C.c_int, C.c_void_p, C.c_void_p]
    return _xs


def dev(a):
    return torch.as_tensor(np.asarray(a, dtype=np.float64), device="cuda")


def noalloc(xs, lines, nu, T, P, sb, Wc, prec, out):
    s = lines.struct()
    st = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    return xs.lib().xs_compute_noalloc(C.byref(s), nu.data_ptr(), nu.numel(), T.data_ptr(), P.data_ptr(), T.numel(),
                                       sb, Wc, prec, out.data_ptr(), st)


@pytest.mark.parametrize("prec", [0, 1])
def test_noalloc_matches_workspace_entry_point_twice(xs, prec):
    lines = xs.DeviceLines(W.water_like(6000, seed=61, nu_min=4345.0, nu_max=4385.0))
    nu = dev(W.grid_lognu(3000, 4355.0, 4375.0))
    P = dev([1e-3, 0.3, 30.0])
    T = dev([700.0, 1200.0, 1800.0])
    ref = xs.xs_compute(lines, nu, T, P, 1.1, 25.0, prec).double().cpu().numpy()
    dt = torch.float32 if prec == 1 else torch.float64
    for _ in range(2):  # the second call reuses the array the first one left behind
        out = torch.full((3, 3000), float("nan"), dtype=dt, device="cuda")
        assert noalloc(xs, lines, nu, T, P, 1.1, 25.0, prec, out) == 0
        got = out.double().cpu().numpy()
        if prec == 0:
            assert np.allclose(got, ref, rtol=1e-10, atol=0)
        else:
            m = ref > 1e-6 * ref.max()
            assert np.max(np.abs(got[m] - ref[m]) / ref[m]) < 1e-5
            assert np.all(np.isfinite(got))


def test_noalloc_rejects_problems_beyond_its_scratch(xs):
    lines = xs.DeviceLines(W.water_like(2_000_000, seed=62))
    nu = dev(W.grid_lognu(100_000))
    P, T = dev([1.0]), dev([1300.0])
    out = torch.zeros((1, 100_000), dtype=torch.float32, device="cuda")
    assert noalloc(xs, lines, nu, T, P, 1.0, 25.0, 1, out) == -6  # XS_ETOOBIG, nothing launched
    assert not out.any()
