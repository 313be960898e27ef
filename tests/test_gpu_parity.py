"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Binning is compared bit-exactly (index work); spreading and interpolation
within the tolerances of tests/_gpu.py.  Sizes span several tiles and a
ragged tail; the full-size case is the 128^3 MAC grid with 10^6 points in
the launch configuration bench.py times.
"""
import hashlib

import numpy as np
import pytest
import torch

import ib_inputs
from _gpu import FLOOR32, FLOOR64, assert_interp_close, assert_spread_close, dev, host

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    from paper_2012_06646_gb300 import build
    build()
    from paper_2012_06646_gb300.plan import Plan
    return Plan


def _edge_points(n, L, dim, dtype):
    """Cell faces, half cells, box ends, negatives, beyond L, tiny and far (in range) positions."""
    L = np.asarray(L[:dim], dtype=np.float64)
    h = L / np.asarray(n[:dim])
    pts = [np.zeros(dim), h * 3, h * 2.5, L - h * 0.5, -h * 0.25, L + h * 1.5, L * 5.25 + h * 0.125,
           -L * 3 - h * 0.75, np.full(dim, 1e-30), np.full(dim, -1e-30), h * 7 - np.spacing(h * 7),
           np.full(dim, 1e-6)]
    return np.array(pts).astype(dtype)


CASES = [
    # dim, n, L, mac, kernel, ncomp, npts, dtype
    (3, (40, 36, 20), (1.0, 0.9, 0.5), True, 0, 3, 5000, np.float32),
    (3, (32, 32, 32), (1.0, 1.0, 1.0), True, 1, 3, 3000, np.float32),
    (3, (17, 33, 16), (1.0, 1.0, 1.0), False, 0, 1, 2000, np.float32),
    (3, (20, 20, 20), (2.0, 2.0, 2.0), False, 1, 4, 2000, np.float32),
    (3, (24, 20, 28), (0.3, 0.7, 1.1), True, 0, 3, 2000, np.float32),      # scale N/L not short: FP64 cell path
    (3, (96, 8, 12), (16.0, 1.0, 1.5), True, 0, 3, 3000, np.float32),
    (3, (4, 5, 6), (1.0, 1.0, 1.0), True, 0, 3, 300, np.float32),
    (3, (1, 2, 3), (1.0, 1.0, 1.0), False, 0, 1, 100, np.float32),
    (2, (64, 40), (1.0, 0.625), True, 0, 2, 2000, np.float32),
    (2, (70, 33), (1.0, 1.0), False, 1, 3, 2000, np.float32),
    (2, (1, 1), (1.0, 1.0), False, 0, 1, 20, np.float32),
    (2, (64, 64), (1.0, 1.0), False, 0, 2, 1000, np.float64),              # the 2-D FP64 workload
    (3, (24, 24, 24), (1.0, 1.0, 1.0), True, 0, 3, 2000, np.float64),
    (3, (18, 18, 18), (1.0, 1.0, 1.0), True, 1, 3, 500, np.float64),
]


def _case_inputs(dim, n, L, ncomp, npts, dtype, seed):
    X = np.concatenate([ib_inputs.uniform_points(seed, npts, L, dim, dtype=dtype), _edge_points(n, L, dim, dtype)])
    G = ib_inputs.normal_array(seed + 1, (len(X), ncomp), dtype=dtype)
    u = ib_inputs.normal_array(seed + 2, (ncomp,) + tuple(reversed(n[:dim])), dtype=dtype)
    return X, G, u


@pytest.mark.parametrize("case", CASES, ids=[f"{c[0]}d-{'x'.join(map(str, c[1]))}-{'mac' if c[3] else 'cc'}-k{c[4]}"
                                             f"-c{c[5]}-{np.dtype(c[7]).name}" for c in CASES])
def test_bin_spread_interp_match_oracle(P, orc, case):
    dim, n, L, mac, kernel, ncomp, npts, dtype = case
    X, G, u = _case_inputs(dim, n, L, ncomp, npts, dtype, seed=sum(n) + dim)
    tdt = torch.float32 if dtype == np.float32 else torch.float64
    plan = P(dim, n, L, grid="mac" if mac else "cc", kernel="peskin4" if kernel == 0 else "cosine4", dtype=tdt,
             ncomp=ncomp, max_points=len(X))
    g = orc.Grid(dim=dim, n=n, L=L, mac=mac, kernel=kernel, ncomp=ncomp)
    Xd, Gd, ud = dev(X), dev(G), dev(u)

    # binning: exact (index work)
    plan.bin(Xd)
    perm, start = plan.bins()
    key = orc.cell_keys(g, X.astype(np.float64))
    perm_ref, start_ref, _ = orc.bin_stable(key, g.ncell)
    assert np.array_equal(host(perm), perm_ref)
    assert np.array_equal(host(start)[: g.ncell + 1], start_ref)

    f = plan.spread(Xd, Gd, reuse_bins=True)
    U = plan.interpolate(Xd, ud, reuse_bins=True)
    plan.check()
    f_ref, fabs = orc.spread(g, X, G)
    U_ref, Uabs = orc.interp(g, X, u)
    rel, floor = (1e-5, FLOOR32) if dtype == np.float32 else (1e-12, FLOOR64)
    assert_spread_close(host(f), f_ref, fabs, rel, floor)
    assert_interp_close(host(U), U_ref, Uabs, rel, floor)


def test_full_size_128_mac_1e6(P, orc):
    """The benchmark workload: 128^3 MAC grid, 10^6 uniform points, FP32, standard kernel."""
    n, L, npts = (128, 128, 128), (1.0, 1.0, 1.0), 1_000_000
    X = ib_inputs.uniform_points(100, npts, L, 3)
    G = ib_inputs.normal_array(101, (npts, 3))
    u = ib_inputs.shear_field_mac(128, 1.0, 1.0) + ib_inputs.normal_array(102, (3, 128, 128, 128))
    plan = P(3, n, L, max_points=npts)
    Xd, Gd, ud = dev(X), dev(G), dev(u)
    plan.bin(Xd)
    f = plan.spread(Xd, Gd, reuse_bins=True)
    U = plan.interpolate(Xd, ud, reuse_bins=True)
    plan.check()
    g = orc.Grid(dim=3, n=n, L=L, mac=True)
    f_ref, fabs = orc.spread(g, X, G)
    assert_spread_close(host(f), f_ref, fabs)
    del f_ref, fabs
    U_ref, Uabs = orc.interp(g, X, u)
    assert_interp_close(host(U), U_ref, Uabs)
    perm, start = plan.bins()
    perm_ref, start_ref, _ = orc.bin_stable(orc.cell_keys(g, X.astype(np.float64)), g.ncell)
    assert np.array_equal(host(perm), perm_ref)
    assert np.array_equal(host(start)[: g.ncell + 1], start_ref)


def test_bit_reproducible_over_runs(P):
    n, npts = (128, 128, 128), 1_000_000
    X = dev(ib_inputs.uniform_points(7, npts, (1.0, 1.0, 1.0), 3))
    G = dev(ib_inputs.normal_array(8, (npts, 3)))
    u = dev(ib_inputs.normal_array(9, (3, 128, 128, 128)))
    plan = P(3, n, (1.0, 1.0, 1.0), max_points=npts)
    hashes = set()
    for _ in range(10):
        f = plan.spread(X, G)
        U = plan.interpolate(X, u, reuse_bins=True)
        h = hashlib.sha256(host(f).tobytes() + host(U).tobytes()).hexdigest()
        hashes.add(h)
    assert len(hashes) == 1


def test_accumulate_and_empty(P, orc):
    n = (20, 24, 28)
    plan = P(3, n, (1.0, 1.0, 1.0), max_points=500)
    X = ib_inputs.uniform_points(3, 500, (1.0, 1.0, 1.0), 3)
    G = ib_inputs.normal_array(4, (500, 3))
    f0 = ib_inputs.normal_array(5, plan.grid_shape())
    fd = dev(f0.copy())
    plan.spread(dev(X), dev(G), f=fd, accumulate=True)
    f_ref, fabs = orc.spread(orc.Grid(dim=3, n=n, L=(1.0, 1.0, 1.0)), X, G)
    out = host(fd).astype(np.float64)
    err = np.abs(out - (f0 + f_ref))
    assert np.all(err <= 1e-5 * (fabs + np.abs(f0)) + 2 * np.spacing(np.abs(f0).astype(np.float32)) + FLOOR32)
    # no points: overwrite gives zeros, accumulate leaves f untouched, interpolation writes nothing
    empty = dev(np.zeros((0, 3), np.float32))
    z = plan.spread(empty, dev(np.zeros((0, 3), np.float32)), f=dev(f0.copy()))
    assert not host(z).any()
    keep = plan.spread(empty, dev(np.zeros((0, 3), np.float32)), f=dev(f0.copy()), accumulate=True)
    assert np.array_equal(host(keep), f0)
    assert plan.interpolate(empty, dev(f0)).shape == (0, 3)


def test_reuse_bins_requires_matching_bin(P):
    from paper_2012_06646_gb300._abi import IB_ERR_NO_BINS, IBError
    plan = P(3, (16, 16, 16), (1.0, 1.0, 1.0), max_points=100)
    X = dev(ib_inputs.uniform_points(1, 100, (1.0, 1.0, 1.0), 3))
    X2 = X.clone()
    plan.bin(X)
    plan.interpolate(X, dev(np.zeros(plan.grid_shape(), np.float32)), reuse_bins=True)
    with pytest.raises(IBError) as e:
        plan.interpolate(X2, dev(np.zeros(plan.grid_shape(), np.float32)), reuse_bins=True)
    assert e.value.status == IB_ERR_NO_BINS


def test_nonfinite_and_out_of_range_positions_are_reported(P, orc):
    from paper_2012_06646_gb300._abi import IB_ERR_NONFINITE, IB_ERR_RANGE, IBError
    n = (16, 16, 16)
    plan = P(3, n, (1.0, 1.0, 1.0), max_points=64)
    X = ib_inputs.uniform_points(2, 64, (1.0, 1.0, 1.0), 3)
    G = ib_inputs.normal_array(3, (64, 3))
    u = ib_inputs.normal_array(4, plan.grid_shape())
    Xbad = X.copy()
    Xbad[5, 1] = np.nan
    Xbad_d = dev(Xbad)                 # one device array: reuse_bins requires the X that was binned
    f = plan.spread(Xbad_d, dev(G))
    U = plan.interpolate(Xbad_d, dev(u), reuse_bins=True)
    with pytest.raises(IBError) as e:
        plan.check()
    assert e.value.status == IB_ERR_NONFINITE
    plan.check()  # the error word was cleared
    keep = np.ones(64, bool)
    keep[5] = False
    g = orc.Grid(dim=3, n=n, L=(1.0, 1.0, 1.0))
    f_ref, fabs = orc.spread(g, X[keep], G[keep])
    assert_spread_close(host(f), f_ref, fabs)
    Uh = host(U)
    assert np.isnan(Uh[5]).all() and np.isfinite(Uh[keep]).all()
    Xfar = X.copy()
    Xfar[0, 0] = 1e8   # 1e8 * 16 cells > 2^30
    plan.interpolate(dev(Xfar), dev(u))
    with pytest.raises(IBError) as e:
        plan.check()
    assert e.value.status == IB_ERR_RANGE


def test_positions_changed_after_binning_are_reported(P):
    from paper_2012_06646_gb300._abi import IB_ERR_BINS_STALE, IBError
    n = (32, 32, 32)
    plan = P(3, n, (1.0, 1.0, 1.0), max_points=500)
    X = ib_inputs.uniform_points(21, 500, (1.0, 1.0, 1.0), 3)
    G = ib_inputs.normal_array(22, (500, 3))
    u = ib_inputs.normal_array(23, plan.grid_shape())
    Xd, Gd, ud = dev(X), dev(G), dev(u)
    plan.bin(Xd)
    f_ok = plan.spread(Xd, Gd, reuse_bins=True)
    plan.check()
    Xd[7] = torch.tensor([(X[7, 0] + 0.5) % 1.0, X[7, 1], X[7, 2]], dtype=torch.float32)   # another tile
    f = plan.spread(Xd, Gd, reuse_bins=True)
    U = plan.interpolate(Xd, ud, reuse_bins=True)
    with pytest.raises(IBError) as e:
        plan.check()
    assert e.value.status == IB_ERR_BINS_STALE
    Uh = host(U)
    assert np.isnan(Uh[7]).all() and np.isfinite(np.delete(Uh, 7, axis=0)).all()
    # the moved point contributes nothing; every other contribution is as before
    Xk = X.copy()
    Gk = G.copy()
    Gk[7] = 0.0
    plan.bin(dev(Xk))
    f_ref = plan.spread(dev(Xk), dev(Gk), reuse_bins=False)
    assert np.allclose(host(f), host(f_ref), rtol=1e-5, atol=1e-5 * float(np.abs(host(f_ok)).max()))
    plan.check()


@pytest.mark.parametrize("per_cell", [None, 8832], ids=["rbc2562", "rbc8832"])
def test_compensated_spread_on_membranes(P, orc, per_cell):
    """Clustered RBC membranes: 17 red cells compressed to about 40 % volume
    fraction in the 128^3 MAC box (2562 points per cell, and the paper's 8832),
    FP32 with TwoSum node sums and plain; interpolation on the same points."""
    mem = ib_inputs.pack_membranes(0, points_per_cell=per_cell)
    assert len(mem.centres) == 17 and mem.volume_fraction > 0.385
    X = mem.X
    G = ib_inputs.membrane_forces(0, mem)
    n = (128, 128, 128)
    u = ib_inputs.normal_array(7, (3, 128, 128, 128))
    plan = P(3, n, (1.0, 1.0, 1.0), max_points=len(X), compensated=True)
    g = orc.Grid(dim=3, n=n, L=(1.0, 1.0, 1.0))
    f_ref, fabs = orc.spread(g, X, G)
    fc = host(plan.spread(dev(X), dev(G), compensated=True))
    fp = host(plan.spread(dev(X), dev(G), reuse_bins=True))
    U = host(plan.interpolate(dev(X), dev(u), reuse_bins=True))
    plan.check()
    assert_spread_close(fc, f_ref, fabs, what="compensated")
    assert_spread_close(fp, f_ref, fabs, what="plain")
    U_ref, Uabs = orc.interp(g, X, u)
    assert_interp_close(U, U_ref, Uabs)
    ec = np.abs(fc - f_ref).sum()
    ep = np.abs(fp - f_ref).sum()
    assert ec <= ep


def test_pos_grad_matches_oracle(P, orc):
    n, npts = (20, 16, 24), 800
    plan = P(3, n, (1.0, 0.8, 1.2), max_points=npts)
    g = orc.Grid(dim=3, n=n, L=(1.0, 0.8, 1.2))
    X = ib_inputs.uniform_points(11, npts, g.L, 3)
    field = ib_inputs.normal_array(12, plan.grid_shape())
    v = ib_inputs.normal_array(13, (npts, 3))
    D = host(plan.pos_grad(dev(X), dev(field), dev(v), scale=2.5))
    D_ref, Dabs = orc.pos_grad(g, X, field, v)
    assert_interp_close(D, 2.5 * D_ref, 2.5 * Dabs, rel=2e-5, what="pos_grad")
    # IB_SPREAD_GRAD: the library applies spreading's h^-d to the same sum
    hmd = orc.inv_cell_volume(g)
    Ds = host(plan.pos_grad(dev(X), dev(field), dev(v), scale=2.5, reuse_bins=True, spread=True))
    assert_interp_close(Ds, 2.5 * hmd * D_ref, 2.5 * hmd * Dabs, rel=2e-5, what="pos_grad (spread)")


def test_advect_wraps(P):
    plan = P(3, (32, 32, 32), (1.0, 2.0, 0.5), max_points=1000)
    X = ib_inputs.uniform_points(21, 1000, (1.0, 2.0, 0.5), 3)
    U = ib_inputs.normal_array(22, (1000, 3)) * np.float32(20.0)
    dt = 0.01
    out = host(plan.advect(dev(X), dev(U), dt))
    want = X.astype(np.float64) + dt * U.astype(np.float64)
    L = np.array([1.0, 2.0, 0.5])
    want = want - L * np.floor(want / L)
    d = np.abs(out - want)
    d = np.minimum(d, L - d)                 # distance on the circle
    assert np.all(d <= 4 * np.spacing(np.float32(2.0)))
    assert np.all((out >= 0) & (out <= L))
