"""z-slab decomposition on one GPU: the slabs of a z-split, each with its own
plan, its own points (routed by ib_slab_owner) and a halo exchange with its
neighbours, must give the single plan's spread and interpolation bit for bit
(every node sum over the same boxes in the same order; every point's
interpolation from the same staged values).  The planes a slab does not own
or receive are NaN in its field, so interpolation proves the halo suffices."""
import numpy as np
import pytest
import torch

import ib_inputs
from _gpu import assert_spread_close, dev, host

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mods():
    from paper_2012_06646_gb300 import build
    build()
    from paper_2012_06646_gb300 import slab
    from paper_2012_06646_gb300.plan import Plan
    return Plan, slab


def _points(seed, npts, n, L, dtype):
    X = ib_inputs.uniform_points(seed, npts, L, 3, dtype=np.float64)
    h = L[2] / n[2]
    k = npts // 4                                   # a quarter of the points within a cell of a slab boundary
    planes = np.arange(0, n[2] + 1, 8) * h
    pick = ib_inputs.uniform(ib_inputs.stream_key(seed, "boundary"), k)
    X[:k, 2] = planes[(pick * len(planes)).astype(np.int64) % len(planes)] + (pick - 0.5) * 2.0 * h
    X[:k, 2] = np.mod(X[:k, 2], L[2])
    return X.astype(dtype)


CASES = [
    # n, L, mac, dtype, nslab, compensated
    ((40, 32, 48), (1.0, 0.8, 1.2), True, np.float32, 2, False),
    ((40, 32, 48), (1.0, 0.8, 1.2), True, np.float32, 3, True),
    ((24, 24, 48), (1.0, 1.0, 2.0), True, np.float32, 6, False),     # one tile layer per slab
    ((33, 20, 32), (1.0, 0.6, 1.0), False, np.float32, 2, False),    # cell-centred, odd n0
    ((24, 16, 32), (1.0, 1.0, 1.0), True, np.float64, 4, False),
]


@pytest.mark.parametrize("case", CASES, ids=[f"{'x'.join(map(str, c[0]))}-{'mac' if c[2] else 'cc'}-"
                                             f"{np.dtype(c[3]).name}-s{c[4]}{'-comp' if c[5] else ''}" for c in CASES])
def test_slabs_equal_the_single_plan_bit_for_bit(mods, case):
    Plan, slab = mods
    n, L, mac, dtype, nslab, comp = case
    tdt = torch.float32 if dtype == np.float32 else torch.float64
    npts = 20_000
    X = _points(sum(n) + nslab, npts, n, L, dtype)
    G = ib_inputs.normal_array(5, (npts, 3), dtype=dtype)
    u = ib_inputs.normal_array(6, (3, n[2], n[1], n[0]), dtype=dtype)
    Xd, Gd, ud = dev(X), dev(G), dev(u)
    kw = dict(grid="mac" if mac else "cc", dtype=tdt, ncomp=3, compensated=comp)
    whole = Plan(3, n, L, max_points=npts, **kw)
    f_ref = whole.spread(Xd, Gd, compensated=comp)
    U_ref = whole.interpolate(Xd, ud, reuse_bins=True)
    whole.check()

    bounds = slab.layer_bounds(n[2] // 8, nslab)
    owner = slab.owners(whole, Xd, bounds)
    assert bool((owner >= 0).all())
    cz = np.floor(X[:, 2].astype(np.float64) * (n[2] / L[2])).astype(np.int64) % n[2]
    want_owner = np.searchsorted(np.array(bounds) * 8, cz, side="right") - 1
    assert np.array_equal(host(owner), want_owner)     # the exact cell's tile layer
    plans, slabs, parts, xs = [], [], [], []
    for k in range(nslab):
        idx = torch.nonzero(owner == k).flatten()
        p = Plan(3, n, L, max_points=max(1, len(idx)), **kw)
        s = slab.Slab(p, k, bounds, compensated=comp)
        Xk = Xd[idx].contiguous()
        s.spread(Xk, Gd[idx].contiguous())
        plans.append(p)
        slabs.append(s)
        parts.append(idx)
        xs.append(Xk)
    slab.exchange_local(slabs)
    f = torch.full(whole.grid_shape(), float("nan"), dtype=tdt, device="cuda")
    for s in slabs:
        s.combine(f)
    assert torch.equal(f, f_ref)

    # interpolation: each slab's field holds its own planes and the received halo, NaN elsewhere
    fields = []
    for s in slabs:
        uk = torch.full_like(ud, float("nan"))
        z0, z1 = s.planes
        uk[:, z0:z1] = ud[:, z0:z1]
        fields.append(uk)
    slab.exchange_field_local(slabs, fields)
    U = torch.full_like(U_ref, float("nan"))
    for p, idx, Xk, uk in zip(plans, parts, xs, fields):
        U[idx] = p.interpolate(Xk, uk, reuse_bins=True)      # the slab's bins from its spread
        p.check()
    assert torch.equal(U, U_ref)
    for p in plans:
        p.close()
    whole.close()


def test_slab_spread_matches_the_oracle_and_accumulates(mods, orc):
    Plan, slab = mods
    n, L, npts = (32, 24, 32), (1.0, 0.75, 1.0), 8000
    X = _points(3, npts, n, L, np.float32)
    G = ib_inputs.normal_array(8, (npts, 3))
    Xd, Gd = dev(X), dev(G)
    whole = Plan(3, n, L, max_points=npts)
    f0 = dev(ib_inputs.normal_array(9, (3, 32, 24, 32)))
    f_acc_ref = whole.spread(Xd, Gd, f=f0.clone(), accumulate=True)
    bounds = slab.layer_bounds(4, 2)
    owner = slab.owners(whole, Xd, bounds)
    slabs, plans = [], []
    for k in range(2):
        idx = torch.nonzero(owner == k).flatten()
        p = Plan(3, n, L, max_points=len(idx))
        s = slab.Slab(p, k, bounds)
        s.spread(Xd[idx].contiguous(), Gd[idx].contiguous())
        slabs.append(s)
        plans.append(p)
    slab.exchange_local(slabs)
    f = torch.empty_like(f0)
    f_acc = f0.clone()
    for s in slabs:
        s.combine(f)
        s.combine(f_acc, accumulate=True)
    g = orc.Grid(dim=3, n=n, L=L, mac=True)
    f_ref, fabs = orc.spread(g, X, G)
    assert_spread_close(host(f), f_ref, fabs, what="slab spread")
    assert torch.equal(f_acc, f_acc_ref)


def test_slab_arguments_are_checked(mods):
    Plan, slab = mods
    from paper_2012_06646_gb300 import _abi
    p2 = Plan(2, (32, 32), (1.0, 1.0), max_points=10)
    with pytest.raises(_abi.IBError):
        slab.Slab(p2, 0, [0, 4])                          # 2-D plans have no z-slabs
    p = Plan(3, (16, 16, 20), (1.0, 1.0, 1.0), max_points=10)
    with pytest.raises(_abi.IBError):
        slab.Slab(p, 0, [0, 2])                           # n2 not a multiple of 8
    q = Plan(3, (16, 16, 32), (1.0, 1.0, 1.0), max_points=10)
    with pytest.raises(_abi.IBError):
        slab.owners(q, dev(np.zeros((3, 3), np.float32)), [0, 1, 3])   # bounds must end at n2 / 8
