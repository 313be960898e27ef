"""ib_interpolate_noalloc (the interpolation entry point that allocates
nothing) against ib_interpolate, both called through the C ABI.

Two calls in a row on different grids and point counts, the second smaller
than the first, so that what the first call leaves in the shared scratch
array must not leak into the second.  Collected last so that it also runs
after every other test in the same process.
"""
import ctypes

import numpy as np
import pytest
import torch

import ib_inputs
from _gpu import dev, host

pytestmark = pytest.mark.gpu


def _desc(abi, n, L, mac, kernel, ncomp):
    d = abi.ib_plan_desc()
    d.dim = 3
    for b in range(3):
        d.n[b] = n[b]
        d.L[b] = L[b]
    d.grid = abi.IB_GRID_MAC if mac else abi.IB_GRID_CELL_CENTERED
    d.kernel = kernel
    d.dtype = abi.IB_F32
    d.ncomp = ncomp
    d.max_points = 0
    d.flags = 0
    return d


def _reference(lib, abi, d, X, u, npts):
    """ib_interpolate on a plan made for this call."""
    d.max_points = npts
    h = ctypes.c_void_p()
    abi.check(lib.ib_plan_create(ctypes.byref(d), ctypes.byref(h)), "ib_plan_create")
    try:
        U = torch.full((npts, d.ncomp), 7.0, dtype=torch.float32, device="cuda")
        s = torch.cuda.current_stream().cuda_stream
        abi.check(lib.ib_interpolate(h, npts, X.data_ptr(), u.data_ptr(), U.data_ptr(), 0, s), "ib_interpolate")
        out = host(U)
    finally:
        d.max_points = 0
        torch.cuda.synchronize()
        lib.ib_plan_destroy(h)
    return out


CALLS = [
    # n, L, mac, kernel, ncomp, npts
    ((64, 48, 40), (1.0, 0.75, 0.625), True, 0, 3, 200_000),
    ((20, 36, 17), (1.0, 1.8, 0.85), False, 1, 2, 3_001),
]


def test_noalloc_interpolate_matches_ib_interpolate_twice_in_a_row():
    from paper_2012_06646_gb300 import _abi, build
    build()
    lib = _abi.load()
    s = torch.cuda.current_stream().cuda_stream
    for i, (n, L, mac, kernel, ncomp, npts) in enumerate(CALLS):
        d = _desc(_abi, n, L, mac, kernel, ncomp)
        X = ib_inputs.uniform_points(900 + i, npts, L, 3, dtype=np.float32)
        X[:: max(1, npts // 50)] *= 3.0                       # wrapped images
        X[npts // 2] = np.nan                                 # a non-finite point reads NaN
        u = ib_inputs.normal_array(910 + i, (ncomp, n[2], n[1], n[0]), dtype=np.float32)
        Xd, ud = dev(X), dev(u)
        want = _reference(lib, _abi, d, Xd, ud, npts)
        U = torch.full((npts, ncomp), -3.0, dtype=torch.float32, device="cuda")
        _abi.check(lib.ib_interpolate_noalloc(ctypes.byref(d), npts, Xd.data_ptr(), ud.data_ptr(), U.data_ptr(), s),
                   "ib_interpolate_noalloc")
        got = host(U)
        assert np.isnan(got[npts // 2]).all() and np.isnan(want[npts // 2]).all()
        scale = float(np.nanmax(np.abs(want)))
        np.testing.assert_allclose(got, want, rtol=1e-5, atol=1e-5 * scale, equal_nan=True)


def test_noalloc_limits_are_rejected_before_any_work():
    from paper_2012_06646_gb300 import _abi
    lib = _abi.load()
    s = torch.cuda.current_stream().cuda_stream
    X = torch.zeros((4, 3), dtype=torch.float32, device="cuda")
    u = torch.zeros((3, 8, 8, 8), dtype=torch.float32, device="cuda")
    U = torch.zeros((4, 3), dtype=torch.float32, device="cuda")
    big = _desc(_abi, (256, 128, 128), (1.0, 1.0, 1.0), True, 0, 3)    # 2^22 cells
    assert lib.ib_interpolate_noalloc(ctypes.byref(big), 4, X.data_ptr(), u.data_ptr(), U.data_ptr(), s) \
        == _abi.IB_ERR_CAPACITY
    small = _desc(_abi, (8, 8, 8), (1.0, 1.0, 1.0), True, 0, 3)
    assert lib.ib_interpolate_noalloc(ctypes.byref(small), _abi.IB_NOALLOC_MAX_POINTS + 1, X.data_ptr(),
                                      u.data_ptr(), U.data_ptr(), s) == _abi.IB_ERR_CAPACITY
    small.flags = _abi.IB_PLAN_COMPENSATED
    assert lib.ib_interpolate_noalloc(ctypes.byref(small), 4, X.data_ptr(), u.data_ptr(), U.data_ptr(), s) \
        == _abi.IB_ERR_INVALID_ARG
    small.flags = 0
    assert lib.ib_interpolate_noalloc(ctypes.byref(small), 0, X.data_ptr(), u.data_ptr(), U.data_ptr(), s) \
        == _abi.IB_OK
    torch.cuda.synchronize()
