"""Pins of the oracle on grids with non-periodic ("bounded") dimensions
(Section 3.1: the grid indexing function returns the empty marker outside the
domain, so those nodes take no part).

Independent references: the dense operator of tests/_dense.py without
periodic images along the bounded dimensions; the periodic oracle for points
far from the walls; and closed forms at a wall: a point on the face x = 0 of
a cell-centred grid keeps exactly half its force (the kernel is even and sums
to one), and on the MAC component normal to the wall, whose node sits on the
face, it keeps (1 + phi(0)) / 2.
"""
import numpy as np
import pytest

import ib_inputs
from _dense import dense_S


def _stagger(mac, a, b):
    return (0.0 if a == b else 0.5) if mac else 0.5


CASES = [
    # dim, n, L, mac, kernel, ncomp, bounded
    (2, (6, 5), (1.0, 0.8), True, 0, 2, (True, False)),
    (2, (7, 4), (1.0, 1.0), False, 1, 1, (True, True)),
    (3, (5, 6, 4), (1.0, 1.2, 0.8), True, 0, 3, (False, False, True)),
    (3, (4, 5, 6), (1.0, 1.0, 1.0), False, 2, 2, (True, False, True)),
    (3, (6, 4, 5), (1.0, 1.0, 1.0), True, 3, 3, (True, True, True)),
]


def _points(n, L, dim, bounded, seed):
    """Random points in the box, plus points on the walls, just inside them, and outside."""
    L = np.asarray(L[:dim], dtype=np.float64)
    h = L / np.asarray(n[:dim])
    X = ib_inputs.uniform_points(seed, 10, tuple(L), dim, dtype=np.float64)
    extra = [np.zeros(dim), L.copy(), h * 0.5, L - h * 0.25, h * 1e-9]
    out = []
    for b in range(dim):
        if bounded[b]:
            p = L / 2
            p[b] = -0.5 * h[b]
            out.append(p.copy())
            p[b] = L[b] + 0.25 * h[b]
            out.append(p.copy())
    return np.concatenate([X, np.array(extra)]), np.array(out).reshape(-1, dim)


@pytest.mark.parametrize("dim,n,L,mac,kernel,ncomp,bounded", CASES)
def test_bounded_equals_dense_operator(orc, dim, n, L, mac, kernel, ncomp, bounded):
    g = orc.Grid(dim=dim, n=n, L=L, mac=mac, kernel=kernel, ncomp=ncomp, bounded=bounded)
    X, Xout = _points(n, L, dim, bounded, seed=sum(n) + kernel)
    G = ib_inputs.normal_array(5, (len(X), ncomp), dtype=np.float64)
    u = ib_inputs.normal_array(6, g.shape(), dtype=np.float64)
    f, fabs = orc.spread(g, X, G)
    U, _ = orc.interp(g, X, u)
    h_d = 1.0 / orc.inv_cell_volume(g)
    for a in range(ncomp):
        xi = [_stagger(mac, a, b) for b in range(dim)]
        S = dense_S(n[:dim], L[:dim], xi, kernel, X, bounded)
        fa = S @ G[:, a]
        assert np.max(np.abs(f[a].ravel() - fa)) <= 1e-13 * max(1.0, np.max(np.abs(fa)))
        Ua = h_d * S.T @ u[a].ravel()
        assert np.max(np.abs(U[:, a] - Ua)) <= 1e-13 * max(1.0, np.max(np.abs(Ua)))
    # points outside the domain along a bounded dimension spread nothing and interpolate to NaN
    f2, _ = orc.spread(g, np.concatenate([X, Xout]), np.concatenate([G, np.ones((len(Xout), ncomp))]))
    assert np.array_equal(f2, f)
    U2, _ = orc.interp(g, Xout, u)
    assert np.isnan(U2).all()


@pytest.mark.parametrize("kernel", [0, 1, 2, 3])
def test_interior_points_as_periodic(orc, kernel):
    n, L = (16, 12, 10), (1.0, 0.75, 0.625)
    h = np.array(L) / np.array(n)
    X = 4 * h + ib_inputs.uniform_points(9, 200, tuple(np.array(L) - 8 * h), 3, dtype=np.float64)
    G = ib_inputs.normal_array(10, (200, 3), dtype=np.float64)
    u = ib_inputs.normal_array(11, (3, 10, 12, 16), dtype=np.float64)
    per = orc.Grid(dim=3, n=n, L=L, mac=True, kernel=kernel)
    bnd = orc.Grid(dim=3, n=n, L=L, mac=True, kernel=kernel, bounded=(True, True, True))
    assert np.array_equal(orc.spread(per, X, G)[0], orc.spread(bnd, X, G)[0])
    assert np.array_equal(orc.interp(per, X, u)[0], orc.interp(bnd, X, u)[0])


@pytest.mark.parametrize("kernel", [0, 1, 2, 3])
def test_wall_point_keeps_half_or_more(orc, kernel):
    """x-walls only: a point on x = 0 (and on x = L) keeps 1/2 of its force on the cell-centred grid and
    (1 + phi(0)) / 2 on the wall-normal MAC component; the tangential MAC components keep 1/2."""
    n, L = (8, 6, 6), (1.0, 0.75, 0.75)
    G = np.array([[1.0, 2.0, -3.0]])
    for x in (0.0, 1.0):
        X = np.array([[x, 0.3, 0.4]])
        cc = orc.Grid(dim=3, n=n, L=L, mac=False, kernel=kernel, ncomp=3, bounded=(True, False, False))
        f, _ = orc.spread(cc, X, G)
        tot = f.reshape(3, -1).sum(1) / orc.inv_cell_volume(cc)
        assert np.allclose(tot, 0.5 * G[0], atol=1e-14)
        mac = orc.Grid(dim=3, n=n, L=L, mac=True, kernel=kernel, bounded=(True, False, False))
        f, _ = orc.spread(mac, X, G)
        tot = f.reshape(3, -1).sum(1) / orc.inv_cell_volume(mac)
        # component 0 sits on the faces x = i h: at x = 0 node 0 is in the domain, at x = L node n is not
        keep0 = (1.0 + orc.phi(kernel, 0.0)[0]) / 2 if x == 0.0 else (1.0 - orc.phi(kernel, 0.0)[0]) / 2
        assert tot[0] == pytest.approx(keep0 * G[0, 0], abs=1e-14)
        assert np.allclose(tot[1:], 0.5 * G[0, 1:], atol=1e-14)


@pytest.mark.parametrize("mac", [True, False])
def test_bounded_position_gradients_match_central_differences(orc, mac):
    """Walls in x and z; points within the support of a wall (at least 4 eps inside): the analytic
    gradient of loss = sum(v . U(X)) against FP64 central differences, eps = 1e-6."""
    n, L = (12, 10, 8), (1.0, 0.8, 0.64)
    bounded = (True, False, True)
    g = orc.Grid(dim=3, n=n, L=L, mac=mac, bounded=bounded, ncomp=3)
    h = np.array(L) / np.array(n)
    X = ib_inputs.uniform_points(51, 120, L, 3, dtype=np.float64)
    X[:40, 0] = 1e-4 + 1.9 * h[0] * ib_inputs.uniform_points(52, 40, (1.0,), 1, dtype=np.float64)[:, 0]
    X[40:80, 2] = L[2] - 1e-4 - 1.9 * h[2] * ib_inputs.uniform_points(53, 40, (1.0,), 1, dtype=np.float64)[:, 0]
    field = ib_inputs.normal_array(54, g.shape(), dtype=np.float64)
    v = ib_inputs.normal_array(55, (120, 3), dtype=np.float64)
    D, _ = orc.pos_grad(g, X, field, v)
    eps = 1e-6
    fd = np.zeros_like(X)
    for b in range(3):
        Xp, Xm = X.copy(), X.copy()
        Xp[:, b] += eps
        Xm[:, b] -= eps
        fd[:, b] = (np.sum(v * orc.interp(g, Xp, field)[0], 1) - np.sum(v * orc.interp(g, Xm, field)[0], 1)) / (2 * eps)
    assert np.max(np.abs(D - fd)) <= 1e-6 * np.max(np.abs(D))
    # outside a wall: NaN
    Xo = np.array([[-1e-3, 0.3, 0.3], [0.5, 0.3, L[2] + 1e-3]])
    assert np.isnan(orc.pos_grad(g, Xo, field, v[:2])[0]).all()
