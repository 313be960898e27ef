"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Nothing here compares the oracle with itself: the values come from the
paper's printed worked examples (tests/golden/), closed forms of the
kernels, the kernel moment identities, an independent dense brute-force
operator (tests/_dense.py), conservation, exactness on constant and linear
fields, the transpose relation S* = S^T (Section 2, Eqs. matrix-interp and
matrix-spread), and central finite differences.  test_mutations_are_caught
plants a mistake in the oracle and checks that some pin fails.
"""
import math

import numpy as np
import pytest

from conftest import read_golden
from _dense import dense_S, phi_bspline6, phi_cos, phi_roma3, phi_std

import ib_inputs


# ----------------------------------------------------------------- kernels --

@pytest.mark.parametrize("kernel", [0, 1])
def test_kernel_closed_forms(orc, kernel):
    """Both 4-point kernels take these values (Peskin 2002, cited in Section 2)."""
    s2 = math.sqrt(2.0)
    cases = {0.0: 0.5, 1.0: 0.25, -1.0: 0.25, 0.5: (2 + s2) / 8, -0.5: (2 + s2) / 8,
             1.5: (2 - s2) / 8, -1.5: (2 - s2) / 8, 2.0: 0.0, -2.0: 0.0, 2.5: 0.0, -3.0: 0.0}
    for r, v in cases.items():
        assert orc.phi(kernel, r)[0] == pytest.approx(v, abs=1e-15), (kernel, r)


def test_kernels_differ_at_quarter(orc):
    # standard: (2.5 + sqrt(1.75)) / 8 ; cosine: (1 + cos(pi/8)) / 4
    assert orc.phi(0, 0.25)[0] == pytest.approx(0.47785945694, abs=1e-11)
    assert orc.phi(1, 0.25)[0] == pytest.approx(0.48096988312, abs=1e-11)


R_GRID = np.linspace(0.0, 1.0, 1001, endpoint=False)


def _moments(orc, kernel):
    t = np.array([-1.0, 0.0, 1.0, 2.0])
    w = np.stack([orc.phi(kernel, tt - R_GRID) for tt in t])    # (4, nr)
    return t, w


def test_standard_kernel_identities(orc):
    """Partition of unity, even/odd sums 1/2, zero first moment, sum of squares 3/8."""
    t, w = _moments(orc, 0)
    assert np.max(np.abs(w.sum(0) - 1.0)) < 1e-14
    assert np.max(np.abs(w[[0, 2]].sum(0) - 0.5)) < 1e-14
    assert np.max(np.abs(w[[1, 3]].sum(0) - 0.5)) < 1e-14
    assert np.max(np.abs(((t[:, None] - R_GRID[None, :]) * w).sum(0))) < 1e-14
    assert np.max(np.abs((w ** 2).sum(0) - 0.375)) < 1e-14


def test_cosine_kernel_identities(orc):
    """The cosine kernel keeps partition of unity and sum of squares but not the first moment (Section 2)."""
    t, w = _moments(orc, 1)
    assert np.max(np.abs(w.sum(0) - 1.0)) < 1e-14
    assert np.max(np.abs((w ** 2).sum(0) - 0.375)) < 1e-14
    first = np.max(np.abs(((t[:, None] - R_GRID[None, :]) * w).sum(0)))
    assert 0.02 < first < 0.022


def test_other_width_kernels_closed_forms(orc):
    """3-point kernel (Roma, Peskin, Berger 1999) and the centred quintic B-spline at exact points."""
    roma = {0.0: 2 / 3, 0.5: 0.5, -0.5: 0.5, 1.0: 1 / 6, -1.0: 1 / 6, 1.5: 0.0, 2.0: 0.0,
            0.25: (1 + math.sqrt(1 - 3 / 16)) / 3}
    for r, v in roma.items():
        assert orc.phi(2, r)[0] == pytest.approx(v, abs=1e-15), r
    bsp = {0.0: 11 / 20, 0.5: 841 / 1920, -0.5: 841 / 1920, 1.0: 13 / 60, -1.0: 13 / 60, 1.5: 237 / 3840,
           2.0: 1 / 120, -2.0: 1 / 120, 2.5: 1 / 3840, 3.0: 0.0, -3.5: 0.0}
    for r, v in bsp.items():
        assert orc.phi(3, r)[0] == pytest.approx(v, abs=1e-15), r
    assert [orc.width(k) for k in range(4)] == [4, 4, 3, 6]


def _moments_w(orc, kernel, lo, hi):
    t = np.arange(lo, hi + 1, dtype=np.float64)
    w = np.stack([orc.phi(kernel, tt - R_GRID) for tt in t])
    return t, w


def test_roma3_identities(orc):
    """Partition of unity, zero first moment and sum of squares 1/2 for every offset."""
    t, w = _moments_w(orc, 2, -2, 3)
    d = t[:, None] - R_GRID[None, :]
    assert np.max(np.abs(w.sum(0) - 1.0)) < 1e-14
    assert np.max(np.abs((d * w).sum(0))) < 1e-14
    assert np.max(np.abs((w ** 2).sum(0) - 0.5)) < 1e-14
    assert np.all((w > 0).sum(0) <= 3)                       # at most s = 3 nonzero weights


def test_bspline6_identities(orc):
    """Partition of unity; moments 0, 1/2, 0 of orders 1-3 (the variance of a sum of six unit boxes)."""
    t, w = _moments_w(orc, 3, -3, 4)
    d = t[:, None] - R_GRID[None, :]
    assert np.max(np.abs(w.sum(0) - 1.0)) < 1e-14
    assert np.max(np.abs((d * w).sum(0))) < 1e-14
    assert np.max(np.abs((d * d * w).sum(0) - 0.5)) < 1e-13
    assert np.max(np.abs((d ** 3 * w).sum(0))) < 1e-13
    assert np.all((w > 0).sum(0) <= 6)


def test_other_width_kernels_match_independent_copies(orc):
    r = np.linspace(-3.4, 3.4, 1361)
    assert np.max(np.abs(orc.phi(2, r) - phi_roma3(r))) < 1e-15
    assert np.max(np.abs(orc.phi(3, r) - phi_bspline6(r))) < 1e-15


@pytest.mark.parametrize("kernel", [0, 1, 2, 3])
def test_dphi_closed_forms_and_difference_quotients(orc, kernel):
    """Values at 0, +-1 and the support edge; central differences of phi everywhere (every piece)."""
    edge = {0: 2.0, 1: 2.0, 2: 1.5, 3: 3.0}[kernel]
    # phi'(1): standard -1/2, cosine -pi/8, 3-point -(1 + 0 / q) / 2 = -1/2, B-spline -50/120
    at1 = {0: -0.5, 1: -math.pi / 8, 2: -0.5, 3: -50.0 / 120.0}[kernel]
    assert orc.dphi(kernel, 0.0)[0] == pytest.approx(0.0, abs=1e-15)
    assert orc.dphi(kernel, edge)[0] == pytest.approx(0.0, abs=1e-15)
    assert orc.dphi(kernel, 1.0)[0] == pytest.approx(at1, abs=1e-14)
    assert orc.dphi(kernel, -1.0)[0] == pytest.approx(-at1, abs=1e-14)
    r = np.linspace(-edge - 0.3, edge + 0.3, 461) + 1e-3
    eps = 1e-6
    fd = (orc.phi(kernel, r + eps) - orc.phi(kernel, r - eps)) / (2 * eps)
    assert np.max(np.abs(fd - orc.dphi(kernel, r))) < 1e-6


def test_dense_reference_kernel_copy_matches_closed_forms():
    s2 = math.sqrt(2.0)
    for fn in (phi_std, phi_cos):
        assert fn(np.array([0.0, 1.0, 0.5, 1.5, 2.0])) == pytest.approx(
            [0.5, 0.25, (2 + s2) / 8, (2 - s2) / 8, 0.0], abs=1e-15)


# ---------------------------------------------------- Fig. 1 and Fig. 2 pins --

def test_fig1_cell_points(orc):
    rows = read_golden("fig1_cells.txt")
    pt = [list(map(float, v)) for k, v in rows if k == "point"][0]
    h = float([v for k, v in rows if k == "h"][0][0])
    lo, hi = map(float, [v for k, v in rows if k == "support_box"][0])
    for k, v in rows:
        if k != "stagger":
            continue
        xi = [float(v[0]), float(v[1])]
        want = [float(v[3]), float(v[4])]
        for b in range(2):
            i, r = orc.cell(pt[b], 1.0 / h, xi[b])
            assert h * (i + xi[b]) == pytest.approx(want[b])
            assert 0.0 <= r < 1.0
            # support nodes i + t, t in {-1..2}: exactly the nodes inside the gray box
            nodes = [h * (i + t + xi[b]) for t in (-1, 0, 1, 2)]
            assert all(lo < x < hi for x in nodes)
            assert not (lo < h * (i - 2 + xi[b]) < hi) and not (lo < h * (i + 3 + xi[b]) < hi)


def test_fig2_worked_example(orc):
    rows = dict((k, v) for k, v in read_golden("fig2_worked_example.txt") if k != "point")
    pts = np.array([list(map(float, v[1:])) for k, v in read_golden("fig2_worked_example.txt") if k == "point"])
    nx, ny = int(rows["cells_x"][0]), int(rows["cells_y"][0])
    g = orc.Grid(dim=2, n=(nx, ny), L=(float(nx), float(ny)), mac=False, ncomp=1)
    key = orc.cell_keys(g, pts)
    assert list(key + 1) == [int(v) for v in rows["keys"]]                 # paper numbers keys from 1
    perm, start, q = orc.bin_stable(key, nx * ny)
    assert list(perm + 1) == [int(v) for v in rows["sorted_perm"]]
    assert list(key[perm] + 1) == [int(v) for v in rows["sorted_keys"]]
    assert q == int(rows["q"][0])
    uniq = [k + 1 for k in range(nx * ny) if start[k + 1] > start[k]]
    assert uniq == [int(v) for v in rows["unique_keys"]]


def test_bin_stable_matches_library_stable_sort(orc):
    rng = np.random.default_rng(7)
    key = rng.integers(0, 50, size=2000).astype(np.uint64)
    perm, start, q = orc.bin_stable(key, 50)
    assert np.array_equal(perm, np.argsort(key, kind="stable"))
    assert q == len(np.unique(key))
    assert np.array_equal(start[:-1], np.searchsorted(np.sort(key), np.arange(50)))


# ----------------------------------------------------------- brute force --

def _stagger(mac, a, b):
    return (0.0 if a == b else 0.5) if mac else 0.5


def _edge_points(n, L, dim, seed):
    """Random points plus points exactly on nodes (r = 0), just below a node (r -> 1-),
    on half-cells, and outside [0, L)."""
    h = np.array(L[:dim]) / np.array(n[:dim])
    X = ib_inputs.uniform_points(seed, 12, L, dim, dtype=np.float64)
    extra = [np.zeros(dim), h * 1.0, h * 2.5, np.array(L[:dim]) - 1e-13, -0.3 * h, np.array(L[:dim]) + 0.7 * h]
    extra.append(h * 3 - np.spacing(h * 3))
    return np.concatenate([X, np.array(extra)])


CASES = [
    (2, (5, 4), (1.0, 0.8), False, 0, 2),
    (2, (8, 8), (1.0, 1.0), True, 0, 2),
    (2, (4, 6), (0.7, 1.3), True, 1, 2),
    (2, (3, 2), (1.0, 1.0), False, 1, 1),
    (2, (1, 2), (1.0, 1.0), False, 0, 1),
    (3, (4, 5, 6), (1.0, 1.1, 0.9), True, 0, 3),
    (3, (5, 4, 4), (2.0, 1.0, 1.0), False, 1, 2),
    (3, (2, 3, 4), (1.0, 1.0, 1.0), True, 0, 3),
    (2, (7, 5), (1.0, 0.9), True, 2, 2),
    (2, (6, 9), (1.1, 1.0), False, 3, 2),
    (2, (1, 3), (1.0, 1.0), False, 2, 1),
    (3, (5, 4, 6), (1.0, 0.8, 1.2), True, 2, 3),
    (3, (7, 6, 5), (1.0, 1.0, 0.9), True, 3, 3),
    (3, (2, 3, 4), (1.0, 1.0, 1.0), False, 3, 1),
]


@pytest.mark.parametrize("dim,n,L,mac,kernel,ncomp", CASES)
def test_spread_and_interp_equal_dense_operator(orc, dim, n, L, mac, kernel, ncomp):
    g = orc.Grid(dim=dim, n=n, L=L, mac=mac, kernel=kernel, ncomp=ncomp)
    X = _edge_points(n, L, dim, seed=dim * 100 + sum(n))
    G = ib_inputs.normal_array(3, (len(X), ncomp), dtype=np.float64)
    u = ib_inputs.normal_array(4, g.shape(), dtype=np.float64)
    f, fabs = orc.spread(g, X, G)
    U, _ = orc.interp(g, X, u)
    h_d = 1.0 / orc.inv_cell_volume(g)
    for a in range(ncomp):
        xi = [_stagger(mac, a, b) for b in range(dim)]
        S = dense_S(n[:dim], L[:dim], xi, kernel, X)
        fa = S @ G[:, a]
        assert np.max(np.abs(f[a].ravel() - fa)) <= 1e-13 * max(1.0, np.max(np.abs(fa)))
        Ua = h_d * S.T @ u[a].ravel()
        assert np.max(np.abs(U[:, a] - Ua)) <= 1e-13 * max(1.0, np.max(np.abs(Ua)))
    assert np.all(fabs >= np.abs(f) - 1e-15)


# ------------------------------------------------------------ invariants --

@pytest.mark.parametrize("kernel", [0, 1, 2, 3])
@pytest.mark.parametrize("mac", [True, False])
def test_conservation_of_force(orc, kernel, mac):
    """sum_k f_a[k] h^d = sum_j G_{j,a}, from partition of unity."""
    g = orc.Grid(dim=3, n=(8, 6, 10), L=(0.5, 0.375, 0.625), mac=mac, kernel=kernel, ncomp=3)
    X = ib_inputs.uniform_points(11, 300, g.L, 3, dtype=np.float64)
    G = ib_inputs.normal_array(12, (300, 3), dtype=np.float64)
    f, _ = orc.spread(g, X, G)
    h_d = 1.0 / orc.inv_cell_volume(g)
    tot = f.reshape(3, -1).sum(1) * h_d
    assert np.max(np.abs(tot - G.sum(0))) <= 1e-13 * np.abs(G).sum()


@pytest.mark.parametrize("kernel", [0, 1, 2, 3])
def test_interpolates_constants(orc, kernel):
    g = orc.Grid(dim=3, n=(8, 8, 8), L=(1.0, 1.0, 1.0), mac=True, kernel=kernel)
    X = ib_inputs.uniform_points(21, 200, g.L, 3, dtype=np.float64)
    u = np.ones(g.shape()) * np.array([1.5, -2.0, 0.25])[:, None, None, None]
    U, _ = orc.interp(g, X, u)
    assert np.max(np.abs(U - np.array([1.5, -2.0, 0.25]))) < 1e-14


@pytest.mark.parametrize("kernel", [0, 2, 3])
@pytest.mark.parametrize("mac", [True, False])
def test_interpolates_linears_exactly(orc, mac, kernel):
    """Zero first moment makes the standard, 3-point and B-spline kernels exact on alpha + beta . x
    (away from the periodic seam)."""
    n, L = (16, 12, 20), (1.0, 0.75, 1.25)
    g = orc.Grid(dim=3, n=n, L=L, mac=mac, kernel=kernel)
    h = np.array(L) / np.array(n)
    X = 3 * h + ib_inputs.uniform_points(22, 300, np.array(L) - 6 * h, 3, dtype=np.float64)
    alpha, beta = np.array([0.3, -1.1, 2.0]), np.array([[1.0, -2.0, 0.5], [0.2, 0.7, -1.3], [-0.4, 0.1, 0.9]])
    u = np.zeros(g.shape())
    from _dense import node_positions
    for a in range(3):
        xi = [_stagger(mac, a, b) for b in range(3)]
        pos = node_positions(n, L, xi)
        u[a] = (alpha[a] + pos @ beta[a]).reshape(u[a].shape)
    U, _ = orc.interp(g, X, u)
    want = alpha[None, :] + X @ beta.T
    assert np.max(np.abs(U - want)) < 1e-13


@pytest.mark.parametrize("kernel", [0, 1, 2, 3])
def test_adjointness(orc, kernel):
    """<S G, u>_h = h^d sum_k f_k u_k equals <G, S* u>_L = sum_j G_j U_j (target: 1e-12 relative)."""
    g = orc.Grid(dim=3, n=(12, 10, 8), L=(1.2, 1.0, 0.8), mac=True, kernel=kernel)
    X = ib_inputs.uniform_points(31, 500, g.L, 3, dtype=np.float64)
    G = ib_inputs.normal_array(32, (500, 3), dtype=np.float64)
    u = ib_inputs.normal_array(33, g.shape(), dtype=np.float64)
    f, _ = orc.spread(g, X, G)
    U, _ = orc.interp(g, X, u)
    lhs = np.sum(f * u) / orc.inv_cell_volume(g)
    rhs = np.sum(G * U)
    assert abs(lhs - rhs) <= 1e-12 * max(abs(rhs), np.sum(np.abs(G * U)))


def test_single_point_on_a_node(orc):
    """r = 0: weights are the outer product of (1/4, 1/2, 1/4, 0)."""
    n, L = (6, 6, 6), (0.6, 0.6, 0.6)
    g = orc.Grid(dim=3, n=n, L=L, mac=False, ncomp=1)
    h = 0.1
    X = np.array([[h * (2 + 0.5), h * (3 + 0.5), h * (1 + 0.5)]])     # the cell-centred node (2, 3, 1)
    f, _ = orc.spread(g, X, np.array([[2.0]]))
    w1 = {-1: 0.25, 0: 0.5, 1: 0.25, 2: 0.0}
    want = np.zeros((6, 6, 6))
    for tz in w1:
        for ty in w1:
            for tx in w1:
                want[(1 + tz) % 6, (3 + ty) % 6, (2 + tx) % 6] += 2.0 * w1[tx] * w1[ty] * w1[tz] / h ** 3
    assert np.max(np.abs(f[0] - want)) < 1e-9


# -------------------------------------------------------------- gradients --

@pytest.mark.parametrize("kernel", [0, 1, 2, 3])
def test_position_gradients_match_central_differences(orc, kernel):
    """16^3 MAC grid, 200 points, eps = 1e-6: analytic dLoss/dX against FP64 central differences."""
    g = orc.Grid(dim=3, n=(16, 16, 16), L=(1.0, 1.0, 1.0), mac=True, kernel=kernel)
    X = ib_inputs.uniform_points(41, 200, g.L, 3, dtype=np.float64)
    G = ib_inputs.normal_array(42, (200, 3), dtype=np.float64)
    w = ib_inputs.normal_array(43, g.shape(), dtype=np.float64)
    eps = 1e-6
    # interpolation: loss = sum(v * U(X)), dloss/dX = D(field = w, v)
    D, _ = orc.pos_grad(g, X, w, G)
    fd = np.zeros_like(X)
    for b in range(3):
        Xp, Xm = X.copy(), X.copy()
        Xp[:, b] += eps
        Xm[:, b] -= eps
        fd[:, b] = (np.sum(G * orc.interp(g, Xp, w)[0], 1) - np.sum(G * orc.interp(g, Xm, w)[0], 1)) / (2 * eps)
    assert np.max(np.abs(D - fd)) <= 1e-6 * np.max(np.abs(D))
    # spreading: loss = sum(w * f(X)), dloss/dX_j = h^-d D(field = w, v = G)_j
    Ds = orc.inv_cell_volume(g) * D
    j = np.arange(0, 200, 20)
    fds = np.zeros((len(j), 3))
    for ii, jj in enumerate(j):
        for b in range(3):
            Xp, Xm = X.copy(), X.copy()
            Xp[jj, b] += eps
            Xm[jj, b] -= eps
            fds[ii, b] = (np.sum(w * orc.spread(g, Xp, G)[0]) - np.sum(w * orc.spread(g, Xm, G)[0])) / (2 * eps)
    assert np.max(np.abs(Ds[j] - fds)) <= 1e-6 * np.max(np.abs(Ds))


# ---------------------------------------------------------- mutation check --

def _pins_pass(orc):
    """Re-run a compact set of pins; return False as soon as one fails."""
    try:
        test_conservation_of_force(orc, 0, True)
        test_spread_and_interp_equal_dense_operator(orc, *CASES[5])
        test_spread_and_interp_equal_dense_operator(orc, *CASES[1])
        test_interpolates_linears_exactly(orc, True, 0)
        test_position_gradients_match_central_differences(orc, 0)
    except AssertionError:
        return False
    return True


@pytest.mark.parametrize("mutation", [1, 2, 3, 4])
def test_mutations_are_caught(orc, mutation):
    assert _pins_pass(orc)
    orc.set_mutation(mutation)
    try:
        assert not _pins_pass(orc), f"planted mistake {mutation} went unnoticed"
    finally:
        orc.set_mutation(0)
    assert _pins_pass(orc)


@pytest.mark.parametrize("kernel", [0, 1])
def test_kernel_tail_keeps_relative_accuracy(orc, kernel):
    """Near |r| = 2 the weights vanish like (2 - |r|)^2; the tail must stay accurate relative to itself.
    Leading terms: standard (2-a)^2 / (5 - 2a + sqrt(..)) -> (2-a)^2 / 2; cosine (pi (2-a) / 4)^2 / 2."""
    for eps in (1e-3, 1e-6, 1e-9):
        a = 2.0 - eps
        e = 2.0 - a                                # exact (Sterbenz): the distance actually represented
        lead = e * e / 2.0 if kernel == 0 else (math.pi * e / 4.0) ** 2 / 2.0
        v = orc.phi(kernel, a)[0]
        assert abs(v / lead - 1.0) < 10 * eps + 1e-12, (eps, v, lead)


def test_other_width_kernel_tails_keep_relative_accuracy(orc):
    """3-point: near |r| = 3/2 the weight is (3 - 2a)^2 / (2 (5 - 3a + q)) -> 2 e^2 (e = 3/2 - a);
    B-spline: near |r| = 3 it is e^5 / 120 and near 2 the middle piece tends to 1/120 smoothly."""
    for eps in (1e-3, 1e-6, 1e-9):
        a = 1.5 - eps
        e = 1.5 - a
        v = orc.phi(2, a)[0]
        assert abs(v / (2 * e * e) - 1.0) < 10 * eps + 1e-12, (eps, v)
        a = 3.0 - eps
        e = 3.0 - a
        assert abs(orc.phi(3, a)[0] / (e ** 5 / 120) - 1.0) < 1e-12
        assert abs(orc.phi(3, 2.0 - eps)[0] / phi_bspline6(np.array([2.0 - eps]))[0] - 1.0) < 1e-12
