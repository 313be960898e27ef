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
