"""ib_interpolate_noalloc (the interpolation entry point that allocates
nothing) against ib_interpolate, both called through the C ABI.

Some callers cannot allocate device memory: code whose memory belongs to
another allocator under a fixed budget, and latency-critical loops where
cudaMalloc / cudaFree would synchronise the device.  The entry point serves
them from a fixed array compiled into the library.  Its results must equal
ib_interpolate's bit for bit (the same kernels run on the same bins), on
calls in a row over different grids, dimensions and dtypes, each smaller
than the one before, so that what one call leaves in the shared array
cannot leak into the next.  A second pass repeats the calls and checks that
the device's free memory does not change.  Collected last (file name) so
that it also runs after every other test in the same process.
"""
import ctypes

import numpy as np
import pytest
import torch

import ib_inputs
from _gpu import dev, host

pytestmark = pytest.mark.gpu


def _desc(abi, n, L, mac, kernel, ncomp, dtype):
    d = abi.ib_plan_desc()
    d.dim = len(n)
    for b in range(3):
        d.n[b] = n[b] if b < len(n) else 1
        d.L[b] = L[b] if b < len(n) else 1.0
    d.grid = abi.IB_GRID_MAC if mac else abi.IB_GRID_CELL_CENTERED
    d.kernel = kernel
    d.dtype = abi.IB_F64 if dtype == np.float64 else abi.IB_F32
    d.ncomp = ncomp
    d.max_points = 0
    d.flags = 0
    return d


def _reference(lib, abi, d, X, u, npts, tdtype):
    """ib_interpolate on a plan made for this call."""
    d.max_points = npts
    h = ctypes.c_void_p()
    abi.check(lib.ib_plan_create(ctypes.byref(d), ctypes.byref(h)), "ib_plan_create")
    try:
        U = torch.full((npts, d.ncomp), 7.0, dtype=tdtype, device="cuda")
        s = torch.cuda.current_stream().cuda_stream
        abi.check(lib.ib_interpolate(h, npts, X.data_ptr(), u.data_ptr(), U.data_ptr(), 0, s), "ib_interpolate")
        out = host(U)
    finally:
        d.max_points = 0
        torch.cuda.synchronize()
        lib.ib_plan_destroy(h)
    return out


CALLS = [
    # n, L, mac, kernel, ncomp, npts, dtype -- each call smaller than the one before
    ((64, 48, 40), (1.0, 0.75, 0.625), True, 0, 3, 200_000, np.float32),
    ((300, 200), (1.5, 1.0), False, 0, 2, 20_000, np.float32),         # 2-D, 32 x 32 tiles
    ((20, 36, 17), (1.0, 1.8, 0.85), True, 0, 3, 5_000, np.float64),   # FP64
    ((20, 36, 17), (1.0, 1.8, 0.85), False, 1, 2, 3_001, np.float32),
    ((40, 33), (1.0, 0.825), True, 1, 2, 900, np.float64),             # 2-D FP64
]


def _inputs(i, n, L, ncomp, npts, dtype):
    dim = len(n)
    X = ib_inputs.uniform_points(900 + i, npts, L, dim, dtype=dtype)
    X[:: max(1, npts // 50)] *= 3.0                       # wrapped images
    X[npts // 2] = np.nan                                 # a non-finite point reads NaN
    u = ib_inputs.normal_array(910 + i, (ncomp,) + tuple(reversed(n)), dtype=dtype)
    return dev(X), dev(u)


def _noalloc(lib, abi, d, Xd, ud, npts, ncomp, tdtype):
    s = torch.cuda.current_stream().cuda_stream
    U = torch.full((npts, ncomp), -3.0, dtype=tdtype, device="cuda")
    abi.check(lib.ib_interpolate_noalloc(ctypes.byref(d), npts, Xd.data_ptr(), ud.data_ptr(), U.data_ptr(), s),
              "ib_interpolate_noalloc")
    return U


def test_noalloc_interpolate_equals_ib_interpolate_on_calls_in_a_row():
    from paper_2012_06646_gb300 import _abi, build
    build()
    lib = _abi.load()
    cases = []
    for i, (n, L, mac, kernel, ncomp, npts, dtype) in enumerate(CALLS):
        tdtype = torch.float64 if dtype == np.float64 else torch.float32
        d = _desc(_abi, n, L, mac, kernel, ncomp, dtype)
        Xd, ud = _inputs(i, n, L, ncomp, npts, dtype)
        want = _reference(lib, _abi, d, Xd, ud, npts, tdtype)
        cases.append((d, Xd, ud, npts, ncomp, tdtype, want))
    # first pass: every call in a row, each result bit-identical to ib_interpolate's
    for d, Xd, ud, npts, ncomp, tdtype, want in cases:
        got = host(_noalloc(lib, _abi, d, Xd, ud, npts, ncomp, tdtype))
        assert np.isnan(got[npts // 2]).all() and np.isnan(want[npts // 2]).all()
        assert np.array_equal(got, want, equal_nan=True)
    # second pass, outputs allocated beforehand: the calls change no device memory use
    outs = [torch.full((npts, ncomp), -3.0, dtype=tdtype, device="cuda") for _, _, _, npts, ncomp, tdtype, _ in cases]
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    alloc0 = torch.cuda.memory_allocated()
    s = torch.cuda.current_stream().cuda_stream
    for (d, Xd, ud, npts, ncomp, tdtype, want), U in zip(cases, outs):
        _abi.check(lib.ib_interpolate_noalloc(ctypes.byref(d), npts, Xd.data_ptr(), ud.data_ptr(), U.data_ptr(), s),
                   "ib_interpolate_noalloc")
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    assert torch.cuda.memory_allocated() == alloc0
    for (d, Xd, ud, npts, ncomp, tdtype, want), U in zip(cases, outs):
        assert np.array_equal(host(U), want, equal_nan=True)


def test_noalloc_limits_are_rejected_before_any_work():
    from paper_2012_06646_gb300 import _abi
    lib = _abi.load()
    s = torch.cuda.current_stream().cuda_stream
    X = torch.zeros((4, 3), dtype=torch.float32, device="cuda")
    u = torch.zeros((3, 8, 8, 8), dtype=torch.float32, device="cuda")
    U = torch.zeros((4, 3), dtype=torch.float32, device="cuda")
    big = _desc(_abi, (256, 128, 128), (1.0, 1.0, 1.0), True, 0, 3, np.float32)    # 2^22 cells
    assert lib.ib_interpolate_noalloc(ctypes.byref(big), 4, X.data_ptr(), u.data_ptr(), U.data_ptr(), s) \
        == _abi.IB_ERR_CAPACITY
    big2 = _desc(_abi, (2048, 2048), (1.0, 1.0), True, 0, 2, np.float32)           # 2^22 cells in 2-D
    assert lib.ib_interpolate_noalloc(ctypes.byref(big2), 4, X.data_ptr(), u.data_ptr(), U.data_ptr(), s) \
        == _abi.IB_ERR_CAPACITY
    small = _desc(_abi, (8, 8, 8), (1.0, 1.0, 1.0), True, 0, 3, np.float32)
    assert lib.ib_interpolate_noalloc(ctypes.byref(small), _abi.IB_NOALLOC_MAX_POINTS + 1, X.data_ptr(),
                                      u.data_ptr(), U.data_ptr(), s) == _abi.IB_ERR_CAPACITY
    small.flags = _abi.IB_PLAN_COMPENSATED
    assert lib.ib_interpolate_noalloc(ctypes.byref(small), 4, X.data_ptr(), u.data_ptr(), U.data_ptr(), s) \
        == _abi.IB_ERR_INVALID_ARG
    small.flags = 0
    assert lib.ib_interpolate_noalloc(ctypes.byref(small), 0, X.data_ptr(), u.data_ptr(), U.data_ptr(), s) \
        == _abi.IB_OK
    torch.cuda.synchronize()
