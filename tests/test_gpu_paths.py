"""GPU parity of the kernels' alternative paths, through the C ABI.

Covers ragged point counts (the tail of the four-points-per-thread count
kernel), positions that are not 16-byte aligned (the scalar count kernel and
the scalar position update), the three-component tile kernel on a grid whose
sides are multiples of 8 but unequal, and many invalid positions (handled by
the last block of the interpolation launch).  Binning is compared bit-exactly
with the oracle, spreading and interpolation within the tolerances of
tests/_gpu.py.
"""
import numpy as np
import pytest
import torch

import ib_inputs
from _gpu import assert_interp_close, assert_spread_close, dev, host

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    from paper_2012_06646_gb300 import build
    build()
    from paper_2012_06646_gb300.plan import Plan
    return Plan


def _positions(X, aligned):
    """X on the device, either as its own tensor or 12 bytes past a 16-byte boundary."""
    if aligned:
        return dev(X)
    buf = torch.zeros((X.shape[0] + 1, X.shape[1]), dtype=torch.float32, device="cuda")
    buf[1:] = dev(X)
    Xd = buf[1:]
    assert Xd.data_ptr() % 16 != 0
    return Xd


@pytest.mark.parametrize("aligned", [True, False], ids=["aligned", "unaligned"])
@pytest.mark.parametrize("npts", [1, 1001, 1002, 1003])
def test_ragged_counts_and_unaligned_positions(P, orc, npts, aligned):
    n, L = (40, 24, 32), (1.0, 0.6, 0.8)
    X = ib_inputs.uniform_points(npts, npts, L, 3)
    G = ib_inputs.normal_array(npts + 1, (npts, 3))
    u = ib_inputs.normal_array(npts + 2, (3, 32, 24, 40))
    Xd = _positions(X, aligned)
    plan = P(3, n, L, max_points=npts)
    plan.bin(Xd)
    perm, start = plan.bins()
    g = orc.Grid(dim=3, n=n, L=L, mac=True)
    perm_ref, start_ref, _ = orc.bin_stable(orc.cell_keys(g, X.astype(np.float64)), g.ncell)
    assert np.array_equal(host(perm), perm_ref)
    assert np.array_equal(host(start)[: g.ncell + 1], start_ref)
    f = plan.spread(Xd, dev(G), reuse_bins=True)
    U = plan.interpolate(Xd, dev(u), reuse_bins=True)
    plan.check()
    f_ref, fabs = orc.spread(g, X, G)
    U_ref, Uabs = orc.interp(g, X, u)
    assert_spread_close(host(f), f_ref, fabs)
    assert_interp_close(host(U), U_ref, Uabs)
    # position update in place on the same (possibly unaligned) array: X + dt U wrapped into [0, L)
    dt = 0.05
    Uh = host(U).astype(np.float64)
    plan.advect(Xd, U, dt, out=Xd)
    out = host(Xd).astype(np.float64)
    Lv = np.array(L)
    want = X.astype(np.float64) + dt * Uh
    want = want - Lv * np.floor(want / Lv)
    d = np.abs(out - want)
    d = np.minimum(d, Lv - d)
    assert np.all(d <= 4 * np.spacing(np.float32(1.0)))
    assert np.all((out >= 0) & (out <= Lv))


def test_many_invalid_positions(P, orc):
    from paper_2012_06646_gb300._abi import IB_ERR_NONFINITE, IBError
    n, npts = (32, 32, 32), 5000
    rng = np.random.default_rng(5)
    X = ib_inputs.uniform_points(31, npts, (1.0, 1.0, 1.0), 3)
    G = ib_inputs.normal_array(32, (npts, 3))
    u = ib_inputs.normal_array(33, (3, 32, 32, 32))
    bad = np.zeros(npts, bool)
    bad[rng.choice(npts, 3000, replace=False)] = True
    Xbad = X.copy()
    Xbad[bad, 1] = np.nan
    plan = P(3, n, (1.0, 1.0, 1.0), max_points=npts)
    f = plan.spread(dev(Xbad), dev(G))
    U = plan.interpolate(dev(Xbad), dev(u), reuse_bins=True)
    with pytest.raises(IBError) as e:
        plan.check()
    assert e.value.status == IB_ERR_NONFINITE
    g = orc.Grid(dim=3, n=n, L=(1.0, 1.0, 1.0))
    f_ref, fabs = orc.spread(g, X[~bad], G[~bad])
    assert_spread_close(host(f), f_ref, fabs)
    Uh = host(U)
    assert np.isnan(Uh[bad]).all()
    U_ref, Uabs = orc.interp(g, X[~bad], u)
    assert_interp_close(Uh[~bad], U_ref, Uabs)


SPARSE = [
    # dim, n, mac, ncomp, dtype, compensated
    (3, (48, 40, 32), True, 3, np.float32, False),
    (3, (48, 40, 32), True, 3, np.float32, True),
    (3, (40, 40, 40), False, 2, np.float32, False),
    (3, (24, 32, 40), True, 3, np.float64, False),
    (2, (96, 64), True, 2, np.float32, True),
]


@pytest.mark.parametrize("case", SPARSE, ids=[f"{c[0]}d-{'x'.join(map(str, c[1]))}-{'mac' if c[2] else 'cc'}-c{c[3]}"
                                              f"-{np.dtype(c[4]).name}{'-comp' if c[5] else ''}" for c in SPARSE])
def test_sparse_points_skip_empty_tiles(P, orc, case):
    """Fewer than 8 points per tile: empty tiles write no boxes and the combination
    skips them; points sit in a corner of the box and across the periodic seam."""
    dim, n, mac, ncomp, dtype, comp = case
    L = (1.0,) * dim
    rng_pts = ib_inputs.uniform_points(77, 60, L, dim, dtype=np.float64)
    X = (0.15 * rng_pts - 0.05).astype(dtype)          # a corner cluster, some points at negative coordinates
    X = np.concatenate([X, ib_inputs.uniform_points(78, 5, L, dim, dtype=dtype)])
    G = ib_inputs.normal_array(79, (len(X), ncomp), dtype=dtype)
    tdt = torch.float32 if dtype == np.float32 else torch.float64
    plan = P(dim, n, L, grid="mac" if mac else "cc", dtype=tdt, ncomp=ncomp, max_points=len(X), compensated=comp)
    f = host(plan.spread(dev(X), dev(G), compensated=comp))
    g = orc.Grid(dim=dim, n=n, L=L, mac=mac, ncomp=ncomp)
    f_ref, fabs = orc.spread(g, X, G)
    from _gpu import FLOOR32, FLOOR64
    rel, floor = (1e-5, FLOOR32) if dtype == np.float32 else (1e-12, FLOOR64)
    assert_spread_close(f, f_ref, fabs, rel, floor)
    # a dense call on the same plan afterwards writes every box again
    Xd = ib_inputs.uniform_points(80, 20 * np.prod(n) // 64, L, dim, dtype=dtype)
    Gd = ib_inputs.normal_array(81, (len(Xd), ncomp), dtype=dtype)
    plan2 = P(dim, n, L, grid="mac" if mac else "cc", dtype=tdt, ncomp=ncomp, max_points=len(Xd), compensated=comp)
    fd = host(plan2.spread(dev(Xd), dev(Gd), compensated=comp))
    f_ref2, fabs2 = orc.spread(g, Xd, Gd)
    assert_spread_close(fd, f_ref2, fabs2, rel, floor)


@pytest.mark.parametrize("mac", [True, False], ids=["mac", "cc"])
def test_offsets_near_half_cells_origin_and_negative(P, orc, mac):
    """Positions whose half-staggered offsets are small or whose cell map runs
    through negative or sub-quarter-cell products: half-cell positions and their
    float neighbours, tiny and negative coordinates; each point alone in the box,
    so every node holds a single contribution and its relative error shows."""
    n = (16, 16, 16)
    h = 1.0 / 16
    base = []
    for k in (0, 1, 5):
        for frac in (0.5, 0.25, 0.75, 1e-3, 0.999):
            x = np.float32((k + frac) * h)
            base += [x, np.nextafter(x, np.float32(0)), np.nextafter(x, np.float32(1))]
    base += [np.float32(v) for v in (1e-7, 3e-9, -1e-7, -0.3 * h, -0.5 * h, -0.7 * h, -1.5 * h, -2.5 * h)]
    vals = np.array(base, np.float32)
    for i, x in enumerate(vals):        # one point per call: nodes are never shared
        X = np.array([[x, vals[(i + 7) % len(vals)], vals[(i + 13) % len(vals)]]], np.float32)
        G = np.array([[1.0, -2.0, 0.5]], np.float32)
        plan = P(3, n, (1.0, 1.0, 1.0), grid="mac" if mac else "cc", max_points=1)
        f = host(plan.spread(dev(X), dev(G)))
        g = orc.Grid(dim=3, n=n, L=(1.0, 1.0, 1.0), mac=mac)
        f_ref, fabs = orc.spread(g, X, G)
        assert_spread_close(f, f_ref, fabs, what=f"spread of X = {X[0].tolist()}")


def _bins_ref(orc, g, X):
    return orc.bin_stable(orc.cell_keys(g, X.astype(np.float64)), g.ncell)[:2]


@pytest.mark.parametrize("dtype", [np.float32, np.float64], ids=["f32", "f64"])
def test_binning_in_the_previous_order_stays_exact(P, orc, dtype):
    """A plan re-binning as many points takes them in the order of its last
    bins (consecutive threads then count nearby cells); the bins must still be
    the stable sort, whatever that order: after a small displacement, after a
    new random point set, after invalid positions, and after a binning of a
    different number of points (identity order again)."""
    n, L, npts = (48, 40, 36), (1.0, 0.8, 0.75), 60_000
    g = orc.Grid(dim=3, n=n, L=L, mac=True)
    tdt = torch.float32 if dtype == np.float32 else torch.float64
    plan = P(3, n, L, max_points=npts, dtype=tdt)
    X0 = ib_inputs.uniform_points(31, npts, L, 3, dtype=dtype)
    step = (ib_inputs.normal_array(32, (npts, 3), dtype=np.float64) * (0.3 / 48)).astype(dtype)
    X1 = (X0 + step).astype(dtype)                                   # a timestep's displacement
    X2 = ib_inputs.uniform_points(33, npts, L, 3, dtype=dtype)       # unrelated positions
    X3 = X2.copy()
    X3[::997] = np.nan                                               # invalid positions sort last
    X4 = X1[: npts - 7].copy()                                       # another point count
    for X in (X0, X1, X2, X1, X4, X1):
        plan.bin(dev(X))
        perm, start = plan.bins()
        perm_ref, start_ref = _bins_ref(orc, g, X)
        assert np.array_equal(host(perm), perm_ref)
        assert np.array_equal(host(start)[: g.ncell + 1], start_ref)
        plan.check()
    plan.bin(dev(X3))
    perm, start = plan.bins()
    valid = ~np.isnan(X3).any(axis=1)
    iv, ii = np.flatnonzero(valid), np.flatnonzero(~valid)
    pv, start_ref = _bins_ref(orc, g, X3[valid])
    assert np.array_equal(host(perm), np.concatenate([iv[pv], ii]))  # invalid points last, in index order
    assert np.array_equal(host(start)[: g.ncell + 1], start_ref)
    with pytest.raises(Exception):
        plan.check()                                                 # the NaN positions are reported
    # spreading and interpolation on ordered bins equal those on fresh bins, bit for bit
    G = dev(ib_inputs.normal_array(34, (npts, 3), dtype=dtype))
    u = dev(ib_inputs.normal_array(35, (3, 36, 40, 48), dtype=dtype))
    plan.bin(dev(X0))
    f1 = host(plan.spread(dev(X1), G))                                # bins X1 in X0's order
    U1 = host(plan.interpolate(dev(X1), u, reuse_bins=True))
    fresh = P(3, n, L, max_points=npts, dtype=tdt)
    assert np.array_equal(host(fresh.spread(dev(X1), G)), f1)
    assert np.array_equal(host(fresh.interpolate(dev(X1), u, reuse_bins=True)), U1)


def test_bounded_wait_runs_out_and_the_device_stays_usable(P, orc):
    """The binning scan waits (decoupled look-back) with a bounded number of
    polls; the self-test runs one wait on a chunk state that nothing publishes
    and must report IB_ERR_TIMEOUT, after which binning works as before."""
    from paper_2012_06646_gb300 import _abi
    lib = _abi.load()
    s = torch.cuda.current_stream().cuda_stream
    assert lib.ib_selftest_bounded_wait(s) == _abi.IB_ERR_TIMEOUT
    assert lib.ib_selftest_bounded_wait(s) == _abi.IB_ERR_TIMEOUT
    n, L = (32, 32, 32), (1.0, 1.0, 1.0)
    X = ib_inputs.uniform_points(41, 5000, L, 3)
    plan = P(3, n, L, max_points=5000)
    plan.bin(dev(X))
    plan.check()
    g = orc.Grid(dim=3, n=n, L=L, mac=True)
    perm, start = plan.bins()
    perm_ref, start_ref = _bins_ref(orc, g, X)
    assert np.array_equal(host(perm), perm_ref)
    assert np.array_equal(host(start)[: g.ncell + 1], start_ref)


@pytest.mark.parametrize("comp", [False, True], ids=["plain", "compensated"])
def test_calls_that_overlap_the_previous_one(P, orc, comp):
    """IB_OVERLAP_PREVIOUS: the spreading kernel may start while the interpolation
    before it finishes, and the position update while the spreading's combination
    runs (every kernel of the path is launched programmatically); f and the new
    positions are bit for bit those of the calls issued on their own, eagerly and
    replayed from a CUDA graph, and U is untouched by the overlap."""
    n, L, npts = (48, 40, 56), (1.0, 0.8, 1.1), 150_000
    X = ib_inputs.uniform_points(61, npts, L, 3)
    G = ib_inputs.normal_array(62, (npts, 3))
    u = ib_inputs.normal_array(63, (3, 56, 40, 48))
    Xd, Gd, ud = dev(X), dev(G), dev(u)
    dt = 0.37
    plan = P(3, n, L, max_points=npts, compensated=comp)
    f_alone = plan.spread(Xd, Gd, compensated=comp)
    U_alone = plan.interpolate(Xd, ud, reuse_bins=True)
    Xn_alone = plan.advect(Xd, U_alone, dt)
    f = torch.empty_like(f_alone)
    U = torch.empty_like(U_alone)
    Xn = torch.empty_like(Xn_alone)

    def calls():
        plan.interpolate(Xd, ud, U=U, reuse_bins=True)
        plan.spread(Xd, Gd, f=f, compensated=comp, reuse_bins=True, overlap_previous=True)
        plan.advect(Xd, U, dt, out=Xn, overlap_previous=True)

    def clear():
        for t in (f, U, Xn):
            t.fill_(float("nan"))

    for _ in range(3):
        clear()
        calls()
        assert torch.equal(f, f_alone) and torch.equal(U, U_alone) and torch.equal(Xn, Xn_alone)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        calls()
    torch.cuda.current_stream().wait_stream(s)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        calls()
    for _ in range(3):
        clear()
        g.replay()
        torch.cuda.synchronize()
        assert torch.equal(f, f_alone) and torch.equal(U, U_alone) and torch.equal(Xn, Xn_alone)
    # without IB_REUSE_BINS the flag is ignored by spreading (the call bins first)
    f2 = plan.spread(Xd, Gd, compensated=comp, overlap_previous=True)
    assert torch.equal(f2, f_alone)
    plan.check()
    gd = orc.Grid(dim=3, n=n, L=L, mac=True)
    sel = np.arange(0, npts, 97)
    U_ref, Uabs = orc.interp(gd, X[sel], u)
    assert_interp_close(host(U)[sel], U_ref, Uabs)


def test_flag_arguments_are_checked(P):
    """Bits a call does not take are IB_ERR_INVALID_ARG, before anything is launched; the
    overlap flag is taken by spreading and the position update, and nothing else new."""
    from paper_2012_06646_gb300 import _abi
    npts = 1000
    plan = P(3, (16, 16, 16), (1.0, 1.0, 1.0), max_points=npts)
    X = dev(ib_inputs.uniform_points(5, npts, (1.0, 1.0, 1.0), 3))
    G = dev(ib_inputs.normal_array(6, (npts, 3)))
    f = torch.empty(plan.grid_shape(), dtype=torch.float32, device="cuda")
    U = torch.empty((npts, 3), dtype=torch.float32, device="cuda")
    s = torch.cuda.current_stream().cuda_stream
    lib = plan.lib
    bad = 0x40
    assert lib.ib_spread(plan.handle, npts, X.data_ptr(), G.data_ptr(), f.data_ptr(), bad, s) == _abi.IB_ERR_INVALID_ARG
    assert lib.ib_advect(plan.handle, npts, X.data_ptr(), U.data_ptr(), 0.1, U.data_ptr(), _abi.IB_REUSE_BINS,
                         s) == _abi.IB_ERR_INVALID_ARG
    assert lib.ib_interpolate(plan.handle, npts, X.data_ptr(), f.data_ptr(), U.data_ptr(),
                              _abi.IB_OVERLAP_PREVIOUS, s) == _abi.IB_ERR_INVALID_ARG
    # the accepted forms run
    plan.bin(X)
    plan.spread(X, G, f=f, reuse_bins=True, overlap_previous=True)
    Xn = plan.advect(X, U.zero_(), 0.1, overlap_previous=True)     # spreading wrote neither X nor U
    plan.check()
    assert torch.equal(Xn, X)
