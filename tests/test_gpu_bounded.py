"""Non-periodic ("bounded") dimensions through the C ABI against the FP64
oracle: nodes outside the domain along a bounded dimension take no part
(Section 3.1), positions must lie in [0, L] there (else IB_ERR_RANGE, no
contribution, NaN), and ib_advect does not wrap them.  Tolerances as in
tests/_gpu.py.  The full-size case is a 128^3 MAC channel (walls in z) with
10^6 points; by linearity a 20 000-point sample carries the force.
"""
import numpy as np
import pytest
import torch

import ib_inputs
from _gpu import FLOOR32, FLOOR64, assert_interp_close, assert_spread_close, dev, host

pytestmark = pytest.mark.gpu

KNAMES = {0: "peskin4", 1: "cosine4", 2: "roma3", 3: "bspline6"}


@pytest.fixture(scope="module")
def P():
    from paper_2012_06646_gb300 import build
    build()
    from paper_2012_06646_gb300.plan import Plan
    return Plan


def _wall_points(n, L, dim, bounded, dtype):
    """Points on and next to the walls of the bounded dimensions, inside the domain."""
    L = np.asarray(L[:dim], dtype=np.float64)
    h = L / np.asarray(n[:dim])
    pts = []
    for b in range(dim):
        if not bounded[b]:
            continue
        for v in (0.0, L[b], h[b] * 0.5, h[b] * 1e-7, L[b] - h[b] * 0.25, L[b] - np.spacing(L[b]), h[b] * 1.5):
            p = L * 0.37
            p[b] = v
            pts.append(p)
    P = np.array(pts).astype(dtype)
    # a wall value that rounds above L in the dtype (FP32 1.2 > 1.2) is stepped down to the last
    # position inside the domain (X N/L <= N in FP64, the oracle's test)
    n_ = np.asarray(n[:dim], dtype=np.float64)
    for k in range(len(P)):
        for b in range(dim):
            while P[k, b].astype(np.float64) * (n_[b] / L[b]) > n_[b]:
                P[k, b] = np.nextafter(P[k, b], dtype(-np.inf))
    return P


CASES = [
    # dim, n, L, mac, kernel, ncomp, npts, dtype, bounded
    (3, (24, 20, 28), (1.0, 0.8, 1.2), True, 0, 3, 3000, np.float32, (False, False, True)),
    (3, (12, 10, 9), (1.0, 1.0, 1.0), True, 1, 3, 800, np.float64, (True, True, True)),
    (3, (17, 16, 9), (1.0, 1.0, 1.0), False, 3, 2, 1500, np.float32, (True, True, False)),
    (3, (8, 8, 16), (0.5, 0.5, 1.0), True, 2, 3, 1000, np.float32, (True, False, False)),
    (2, (70, 40), (1.0, 0.625), True, 0, 2, 2000, np.float32, (False, True)),
    (2, (5, 3), (1.0, 1.0), False, 2, 1, 100, np.float64, (True, False)),
]


def _ids(c):
    bd = "".join("xyz"[b] for b in range(c[0]) if c[8][b])
    return f"{c[0]}d-{'x'.join(map(str, c[1]))}-{'mac' if c[3] else 'cc'}-{KNAMES[c[4]]}-{np.dtype(c[7]).name}-b{bd}"


@pytest.mark.parametrize("case", CASES, ids=[_ids(c) for c in CASES])
def test_bounded_matches_oracle(P, orc, case):
    dim, n, L, mac, kernel, ncomp, npts, dtype, bounded = case
    seed = 11 * sum(n) + kernel
    X = np.concatenate([ib_inputs.uniform_points(seed, npts, L, dim, dtype=dtype),
                        _wall_points(n, L, dim, bounded, dtype)])
    G = ib_inputs.normal_array(seed + 1, (len(X), ncomp), dtype=dtype)
    u = ib_inputs.normal_array(seed + 2, (ncomp,) + tuple(reversed(n[:dim])), dtype=dtype)
    tdt = torch.float32 if dtype == np.float32 else torch.float64
    plan = P(dim, n, L, grid="mac" if mac else "cc", kernel=KNAMES[kernel], dtype=tdt, ncomp=ncomp,
             max_points=len(X), bounded=bounded)
    g = orc.Grid(dim=dim, n=n, L=L, mac=mac, kernel=kernel, ncomp=ncomp, bounded=bounded)
    Xd, Gd, ud = dev(X), dev(G), dev(u)
    f = plan.spread(Xd, Gd)
    U = plan.interpolate(Xd, ud, reuse_bins=True)
    plan.check()
    f_ref, fabs = orc.spread(g, X, G)
    U_ref, Uabs = orc.interp(g, X, u)
    rel, floor = (1e-5, FLOOR32) if dtype == np.float32 else (1e-12, FLOOR64)
    assert_spread_close(host(f), f_ref, fabs, rel, floor)
    assert_interp_close(host(U), U_ref, Uabs, rel, floor)
    f2 = plan.spread(Xd, Gd, f=f.clone(), accumulate=True, reuse_bins=True)
    assert_spread_close(host(f2), 2 * f_ref, 2 * fabs, rel, floor)
    plan.close()


def test_bounded_outside_positions_are_reported(P, orc):
    from paper_2012_06646_gb300._abi import IB_ERR_RANGE, IBError
    n, L = (16, 16, 16), (1.0, 1.0, 1.0)
    X = ib_inputs.uniform_points(3, 200, L, 3)
    X[7, 2] = -1e-6                     # below the wall z = 0
    X[9, 2] = 1.0 + 2 ** -20            # above z = L
    X[11, 0] = 1.25                     # outside in x, which is periodic: wrapped, valid
    G = ib_inputs.normal_array(4, (200, 3))
    u = ib_inputs.normal_array(5, (3, 16, 16, 16))
    plan = P(3, n, L, max_points=200, bounded=(False, False, True))
    Xd = dev(X)
    f = plan.spread(Xd, dev(G))
    U = plan.interpolate(Xd, dev(u), reuse_bins=True)
    with pytest.raises(IBError) as e:
        plan.check()
    assert e.value.status == IB_ERR_RANGE
    g = orc.Grid(dim=3, n=n, L=L, mac=True, bounded=(False, False, True))
    f_ref, fabs = orc.spread(g, X, G)
    assert_spread_close(host(f), f_ref, fabs)
    Uh = host(U)
    assert np.isnan(Uh[[7, 9]]).all()
    keep = np.ones(200, bool)
    keep[[7, 9]] = False
    U_ref, Uabs = orc.interp(g, X[keep], u)
    assert_interp_close(Uh[keep], U_ref, Uabs)


def test_bounded_compensated_and_advect(P, orc):
    n, L = (32, 32, 32), (1.0, 1.0, 1.0)
    X = ib_inputs.uniform_points(6, 4000, L, 3)
    G = ib_inputs.normal_array(7, (4000, 3))
    plan = P(3, n, L, max_points=4000, compensated=True, bounded=(False, True, False))
    Xd = dev(X)
    f = plan.spread(Xd, dev(G), compensated=True)
    plan.check()
    g = orc.Grid(dim=3, n=n, L=L, mac=True, bounded=(False, True, False))
    f_ref, fabs = orc.spread(g, X, G)
    assert_spread_close(host(f), f_ref, fabs)
    # advect: periodic dimensions wrap, the bounded one does not
    U = dev(np.tile(np.array([[0.75, 0.75, 0.75]], dtype=np.float32), (4000, 1)))
    Xn = host(plan.advect(Xd, U, 1.0))
    assert np.all((Xn[:, [0, 2]] >= 0) & (Xn[:, [0, 2]] < 1.0))
    assert np.allclose(Xn[:, 1], X[:, 1] + 0.75, atol=1e-6)
    plan.close()


def test_bounded_unsupported_calls(P):
    from paper_2012_06646_gb300 import _abi
    from paper_2012_06646_gb300._abi import IBError
    plan = P(3, (16, 16, 16), (1.0, 1.0, 1.0), max_points=10, bounded=(True, False, False))
    X = dev(ib_inputs.uniform_points(1, 10, (1.0, 1.0, 1.0), 3))
    v = dev(ib_inputs.normal_array(3, (10, 3)))
    with pytest.raises(IBError) as e:
        plan.spread_paper(X, v, algorithm=4)
    assert e.value.status == _abi.IB_ERR_NOT_IMPLEMENTED
    plan.close()


@pytest.mark.parametrize("mac", [True, False])
def test_bounded_pos_grad_matches_oracle(P, orc, mac):
    """Walls in x and z, points on and near the walls included; tolerance as the periodic gradients."""
    from paper_2012_06646_gb300._abi import IB_ERR_RANGE, IBError
    n, L, npts = (20, 16, 24), (1.0, 0.8, 1.2), 800
    bounded = (True, False, True)
    plan = P(3, n, L, grid="mac" if mac else "cc", max_points=npts + 1, bounded=bounded)
    g = orc.Grid(dim=3, n=n, L=L, mac=mac, bounded=bounded)
    X = np.concatenate([ib_inputs.uniform_points(61, npts, L, 3),
                        np.array([[-1e-3, 0.4, 0.6]], dtype=np.float32)])      # outside the x wall
    X[:20, 0] = 0.0
    X[20:40, 2] = np.float32(1.2) - np.float32(2 ** -22)
    field = ib_inputs.normal_array(62, plan.grid_shape())
    v = ib_inputs.normal_array(63, (npts + 1, 3))
    D = host(plan.pos_grad(dev(X), dev(field), dev(v), scale=2.5))
    with pytest.raises(IBError) as e:
        plan.check()
    assert e.value.status == IB_ERR_RANGE
    D_ref, Dabs = orc.pos_grad(g, X, field, v)
    assert np.isnan(D[-1]).all() and np.isnan(D_ref[-1]).all()
    assert_interp_close(D[:-1], 2.5 * D_ref[:-1], 2.5 * Dabs[:-1], rel=2e-5, what="pos_grad")
    plan.close()


def test_bounded_channel_full_size(P, orc):
    """128^3 MAC grid with walls at z = 0 and z = L, 10^6 uniform points, FP32, standard kernel."""
    n, L, npts, ns = (128, 128, 128), (1.0, 1.0, 1.0), 1_000_000, 20_000
    X = ib_inputs.uniform_points(300, npts, L, 3)
    G = np.zeros((npts, 3), dtype=np.float32)
    sample = np.sort(np.random.default_rng(5).choice(npts, ns, replace=False))
    G[sample] = ib_inputs.normal_array(301, (ns, 3))
    u = ib_inputs.normal_array(302, (3, 128, 128, 128))
    plan = P(3, n, L, max_points=npts, bounded=(False, False, True))
    Xd, Gd, ud = dev(X), dev(G), dev(u)
    f = plan.spread(Xd, Gd)
    U = plan.interpolate(Xd, ud, reuse_bins=True)
    plan.check()
    g = orc.Grid(dim=3, n=n, L=L, mac=True, bounded=(False, False, True))
    f_ref, fabs = orc.spread(g, X[sample], G[sample])
    assert_spread_close(host(f), f_ref, fabs)
    U_ref, Uabs = orc.interp(g, X[sample], u)
    assert_interp_close(host(U)[sample], U_ref, Uabs)
