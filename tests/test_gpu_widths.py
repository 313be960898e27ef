"""Kernels of support width s != 4 (the 3-point kernel, s = 3, and the
6-point quintic B-spline, s = 6) through the C ABI, against the FP64 oracle.

Binning is the same as for the 4-point kernels (compared bit-exactly in
test_gpu_parity.py); spreading and interpolation are compared element by
element within the tolerances of tests/_gpu.py (1e-5 of the sum of |terms|
in FP32, 1e-12 in FP64).  The cases span several tiles with ragged tails,
grids smaller than the support (the periodic box wraps a box onto itself
several times) and the edge positions of test_gpu_parity.py.  The full-size
case is the 128^3 MAC grid with 10^6 points: every point goes through the
launch, and by linearity only a sample carries a nonzero force, so the
oracle spreads the sample alone; interpolation is checked on a sample.
"""
import ctypes
import hashlib

import numpy as np
import pytest
import torch

import ib_inputs
from _gpu import FLOOR32, FLOOR64, assert_interp_close, assert_spread_close, dev, host

pytestmark = pytest.mark.gpu

NAMES = {2: "roma3", 3: "bspline6"}


@pytest.fixture(scope="module")
def P():
    from paper_2012_06646_gb300 import build
    build()
    from paper_2012_06646_gb300.plan import Plan
    return Plan


def _edge_points(n, L, dim, dtype):
    L = np.asarray(L[:dim], dtype=np.float64)
    h = L / np.asarray(n[:dim])
    pts = [np.zeros(dim), h * 3, h * 2.5, L - h * 0.5, -h * 0.25, L + h * 1.5, L * 5.25 + h * 0.125,
           -L * 3 - h * 0.75, np.full(dim, 1e-30), np.full(dim, -1e-30), h * 7 - np.spacing(h * 7),
           h * 0.5 + np.spacing(h * 0.5), h * 1.5 - np.spacing(h * 1.5), np.full(dim, 1e-6)]
    return np.array(pts).astype(dtype)


CASES = [
    # dim, n, L, mac, kernel, ncomp, npts, dtype
    (3, (24, 20, 28), (1.0, 0.8, 1.2), True, 2, 3, 3000, np.float32),
    (3, (24, 20, 28), (1.0, 0.8, 1.2), True, 3, 3, 3000, np.float32),
    (3, (17, 16, 9), (1.0, 1.0, 1.0), False, 3, 2, 1500, np.float32),
    (3, (12, 10, 9), (1.0, 1.0, 1.0), True, 2, 3, 800, np.float64),
    (3, (12, 10, 9), (1.0, 1.0, 1.0), True, 3, 3, 800, np.float64),
    (3, (4, 3, 2), (1.0, 1.0, 1.0), True, 3, 3, 200, np.float32),     # grid smaller than the support
    (3, (5, 7, 3), (1.0, 1.0, 1.0), False, 2, 1, 200, np.float64),
    (2, (70, 40), (1.0, 0.625), True, 2, 2, 2000, np.float32),
    (2, (70, 40), (1.0, 0.625), True, 3, 2, 2000, np.float32),
    (2, (33, 65), (1.0, 2.0), False, 3, 4, 1500, np.float64),
    (2, (5, 3), (1.0, 1.0), False, 3, 1, 100, np.float32),
    (2, (1, 4), (1.0, 1.0), False, 2, 1, 50, np.float64),
]


def _ids(c):
    return f"{c[0]}d-{'x'.join(map(str, c[1]))}-{'mac' if c[3] else 'cc'}-{NAMES[c[4]]}-c{c[5]}-{np.dtype(c[7]).name}"


@pytest.mark.parametrize("case", CASES, ids=[_ids(c) for c in CASES])
def test_width_kernels_match_oracle(P, orc, case):
    dim, n, L, mac, kernel, ncomp, npts, dtype = case
    seed = 7 * sum(n) + kernel
    X = np.concatenate([ib_inputs.uniform_points(seed, npts, L, dim, dtype=dtype), _edge_points(n, L, dim, dtype)])
    G = ib_inputs.normal_array(seed + 1, (len(X), ncomp), dtype=dtype)
    u = ib_inputs.normal_array(seed + 2, (ncomp,) + tuple(reversed(n[:dim])), dtype=dtype)
    tdt = torch.float32 if dtype == np.float32 else torch.float64
    plan = P(dim, n, L, grid="mac" if mac else "cc", kernel=NAMES[kernel], dtype=tdt, ncomp=ncomp, max_points=len(X))
    g = orc.Grid(dim=dim, n=n, L=L, mac=mac, kernel=kernel, ncomp=ncomp)
    Xd, Gd, ud = dev(X), dev(G), dev(u)
    f = plan.spread(Xd, Gd)
    U = plan.interpolate(Xd, ud, reuse_bins=True)
    plan.check()
    f_ref, fabs = orc.spread(g, X, G)
    U_ref, Uabs = orc.interp(g, X, u)
    rel, floor = (1e-5, FLOOR32) if dtype == np.float32 else (1e-12, FLOOR64)
    assert_spread_close(host(f), f_ref, fabs, rel, floor)
    assert_interp_close(host(U), U_ref, Uabs, rel, floor)
    # accumulate adds onto what is there
    f2 = plan.spread(Xd, Gd, f=f.clone(), accumulate=True, reuse_bins=True)
    assert_spread_close(host(f2), 2 * f_ref, 2 * fabs, rel, floor)
    plan.close()


@pytest.mark.parametrize("kernel", [2, 3])
def test_width_kernels_full_size(P, orc, kernel):
    """128^3 MAC grid, 10^6 uniform points, FP32; 20000 sampled points carry the force and are interpolated."""
    n, L, npts, ns = (128, 128, 128), (1.0, 1.0, 1.0), 1_000_000, 20_000
    X = ib_inputs.uniform_points(200 + kernel, npts, L, 3)
    G = np.zeros((npts, 3), dtype=np.float32)
    sample = np.sort(np.random.default_rng(kernel).choice(npts, ns, replace=False))
    G[sample] = ib_inputs.normal_array(210 + kernel, (ns, 3))
    u = ib_inputs.normal_array(220 + kernel, (3, 128, 128, 128))
    plan = P(3, n, L, kernel=NAMES[kernel], max_points=npts)
    Xd, Gd, ud = dev(X), dev(G), dev(u)
    f = plan.spread(Xd, Gd)
    U = plan.interpolate(Xd, ud, reuse_bins=True)
    plan.check()
    g = orc.Grid(dim=3, n=n, L=L, mac=True, kernel=kernel)
    f_ref, fabs = orc.spread(g, X[sample], G[sample])
    assert_spread_close(host(f), f_ref, fabs)
    U_ref, Uabs = orc.interp(g, X[sample], u)
    assert_interp_close(host(U)[sample], U_ref, Uabs)
    # bit-reproducible
    h = {hashlib.sha256(host(plan.spread(Xd, Gd)).tobytes()).hexdigest() for _ in range(3)}
    assert h == {hashlib.sha256(host(f).tobytes()).hexdigest()}


def test_width_kernels_unsupported_calls(P):
    from paper_2012_06646_gb300 import _abi
    from paper_2012_06646_gb300._abi import IBError
    plan = P(3, (16, 16, 16), (1.0, 1.0, 1.0), kernel="bspline6", max_points=10)
    X = dev(ib_inputs.uniform_points(1, 10, (1.0, 1.0, 1.0), 3))
    u = dev(ib_inputs.normal_array(2, (3, 16, 16, 16)))
    v = dev(ib_inputs.normal_array(3, (10, 3)))
    with pytest.raises(IBError) as e:
        plan.spread_paper(X, v, algorithm=4)
    assert e.value.status == _abi.IB_ERR_NOT_IMPLEMENTED
    with pytest.raises(IBError) as e:
        P(3, (16, 16, 16), (1.0, 1.0, 1.0), kernel="roma3", max_points=10, compensated=True)
    assert e.value.status == _abi.IB_ERR_INVALID_ARG
    plan.close()


@pytest.mark.parametrize("kernel,bounded", [("roma3", (False, False, False)), ("bspline6", (False, False, False)),
                                            ("bspline6", (True, False, True)), ("peskin4", (True, True, True))])
def test_empty_point_sets(P, kernel, bounded):
    """No points: spreading writes zeros (or leaves f as it was with accumulate), interpolation returns nothing."""
    n = (16, 12, 8)
    plan = P(3, n, (1.0, 1.0, 1.0), kernel=kernel, max_points=10, bounded=bounded)
    X = torch.empty((0, 3), dtype=torch.float32, device="cuda")
    G = torch.empty((0, 3), dtype=torch.float32, device="cuda")
    u = dev(ib_inputs.normal_array(5, (3, 8, 12, 16)))
    f = plan.spread(X, G)
    assert torch.count_nonzero(f).item() == 0
    f0 = dev(ib_inputs.normal_array(6, (3, 8, 12, 16)))
    f2 = plan.spread(X, G, f=f0.clone(), accumulate=True)
    assert torch.equal(f2, f0)
    U = plan.interpolate(X, u)
    plan.check()
    assert tuple(U.shape) == (0, 3)
    plan.close()


GRAD_CASES = [
    # dim, n, L, mac, kernel, dtype, bounded
    (3, (20, 16, 24), (1.0, 0.8, 1.2), True, 2, np.float32, (False, False, False)),
    (3, (20, 16, 24), (1.0, 0.8, 1.2), True, 3, np.float32, (False, False, False)),
    (3, (12, 10, 9), (1.0, 1.0, 1.0), False, 3, np.float64, (False, False, False)),
    (3, (12, 10, 9), (1.0, 1.0, 1.0), True, 2, np.float64, (True, False, True)),
    (2, (40, 24), (1.0, 0.6), True, 3, np.float32, (False, True)),
]


@pytest.mark.parametrize("case", GRAD_CASES, ids=[f"{c[0]}d-{NAMES[c[4]]}-{'mac' if c[3] else 'cc'}-"
                                                   f"{np.dtype(c[5]).name}-b{sum(c[6])}" for c in GRAD_CASES])
def test_width_pos_grad_matches_oracle(P, orc, case):
    dim, n, L, mac, kernel, dtype, bounded = case
    npts = 600
    tdt = torch.float32 if dtype == np.float32 else torch.float64
    plan = P(dim, n, L, grid="mac" if mac else "cc", kernel=NAMES[kernel], dtype=tdt, max_points=npts,
             bounded=bounded)
    g = orc.Grid(dim=dim, n=n, L=L, mac=mac, kernel=kernel, bounded=bounded)
    X = ib_inputs.uniform_points(91 + kernel, npts, L, dim, dtype=dtype)
    field = ib_inputs.normal_array(92, plan.grid_shape(), dtype=dtype)
    v = ib_inputs.normal_array(93, (npts, dim), dtype=dtype)
    D = host(plan.pos_grad(dev(X), dev(field), dev(v), scale=2.5))
    plan.check()
    D_ref, Dabs = orc.pos_grad(g, X, field, v)
    rel, floor = (2e-5, FLOOR32) if dtype == np.float32 else (1e-12, FLOOR64)
    assert_interp_close(D, 2.5 * D_ref, 2.5 * Dabs, rel=rel, floor=floor, what="pos_grad")
    plan.close()


def test_width_autograd_bspline(P, orc):
    """loss = sum(w * spread(G, X)) with the 6-point kernel: dL/dG and dL/dX against the oracle."""
    from paper_2012_06646_gb300 import autograd as ag
    n, npts = (16, 16, 16), 400
    plan = P(3, n, (1.0, 1.0, 1.0), kernel="bspline6", max_points=npts)
    X = ib_inputs.uniform_points(95, npts, (1.0, 1.0, 1.0), 3)
    G = ib_inputs.normal_array(96, (npts, 3))
    w = ib_inputs.normal_array(97, plan.grid_shape())
    Xd = dev(X).requires_grad_(True)
    Gd = dev(G).requires_grad_(True)
    gX, gG = torch.autograd.grad((dev(w) * ag.spread(Xd, Gd, plan)).sum(), (Xd, Gd))
    g = orc.Grid(dim=3, n=n, L=(1.0, 1.0, 1.0), kernel=3)
    hmd = orc.inv_cell_volume(g)
    Uw, Uwabs = orc.interp(g, X, w)
    assert_interp_close(host(gG), hmd * Uw, hmd * Uwabs, what="dL/dG")
    D, Dabs = orc.pos_grad(g, X, w, G)
    assert_interp_close(host(gX), hmd * D, hmd * Dabs, rel=2e-5, what="dL/dX")
    plan.close()
