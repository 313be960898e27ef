"""Pins of the FP64 Stokes oracle (oracle/stokes.py) of the IB step (e).

The oracle solves alpha u + G p - mu L u = alpha u_old + f, D u = 0 on the
periodic MAC grid of Section 2 in Fourier space.  None of these pins uses
its Fourier solve: the reference values come from a dense least-squares solve
of the real-space saddle-point system assembled node by node from the
stencils, the closed form of a shear wave, a force that is a discrete
gradient (no flow), and the stencil residuals.  test_stokes_mutations_caught
plants each of several plausible mistakes in the oracle and checks that a pin
fails.
"""
import numpy as np
import pytest

from oracle import stokes


def _lin(idx, n):
    """Flat index (x fastest) of the grid index tuple idx (per dimension, wrapped)."""
    c, stride = 0, 1
    for b in range(len(n)):
        c += (idx[b] % n[b]) * stride
        stride *= n[b]
    return c


def _nodes(n):
    return [tuple(int(v) for v in np.unravel_index(c, tuple(reversed(n)))[::-1]) for c in range(int(np.prod(n)))]


def _dense_system(n, L, alpha, mu):
    """Saddle-point matrix [[alpha I - mu L, G], [D, 0]], unknowns (u_0..u_{d-1}, p), assembled node by node."""
    dim, N = len(n), int(np.prod(n))
    h = [L[b] / n[b] for b in range(dim)]
    A = np.zeros(((dim + 1) * N, (dim + 1) * N))
    P = dim * N
    for idx in _nodes(n):
        c = _lin(idx, n)
        for a in range(dim):
            row = a * N + c
            A[row, a * N + c] += alpha
            for b in range(dim):
                up = list(idx); up[b] += 1
                dn = list(idx); dn[b] -= 1
                A[row, a * N + _lin(up, n)] -= mu / h[b] ** 2
                A[row, a * N + c] += 2.0 * mu / h[b] ** 2
                A[row, a * N + _lin(dn, n)] -= mu / h[b] ** 2
            dn = list(idx); dn[a] -= 1                       # face a of cell idx sits between cells idx - e_a and idx
            A[row, P + c] += 1.0 / h[a]
            A[row, P + _lin(dn, n)] -= 1.0 / h[a]
        for b in range(dim):                                 # divergence at the cell centre
            up = list(idx); up[b] += 1
            A[P + c, b * N + _lin(up, n)] += 1.0 / h[b]
            A[P + c, b * N + c] -= 1.0 / h[b]
    return A


def _brute(f, n, L, alpha, mu, u_old=None):
    dim, N = len(n), int(np.prod(n))
    g = f if u_old is None else alpha * u_old + f
    rhs = np.concatenate([g[a].ravel() for a in range(dim)] + [np.zeros(N)])
    x = np.linalg.lstsq(_dense_system(n, L, alpha, mu), rhs, rcond=None)[0]
    return np.stack([x[a * N:(a + 1) * N].reshape(tuple(reversed(n))) for a in range(dim)])


def _field(rng, n, zero_mean=False):
    f = rng.standard_normal((len(n),) + tuple(reversed(n)))
    if zero_mean:
        f -= f.mean(axis=tuple(range(1, f.ndim)), keepdims=True)
    return f


CASES = [
    ((5, 4), (1.0, 0.7), 3.0, 0.2, False),
    ((6, 3), (2.0, 1.0), 0.0, 1.5, True),       # steady Stokes (alpha = 0), mean-free force
    ((4, 3, 5), (1.0, 1.3, 0.8), 2.0, 0.5, False),
    ((3, 4, 2), (0.5, 1.0, 0.9), 1.0, 0.0, False),   # mu = 0: the pure projection of g / alpha
    ((4, 4, 3), (1.0, 1.0, 1.0), 0.0, 0.7, True),
]


@pytest.mark.parametrize("n,L,alpha,mu,zero_mean", CASES)
def test_stokes_matches_dense_saddle_point(n, L, alpha, mu, zero_mean):
    rng = np.random.default_rng(sum(n) * 7 + int(10 * alpha))
    f = _field(rng, n, zero_mean)
    u_old = None if alpha == 0.0 else _field(rng, n)
    want = _brute(f, n, L, alpha, mu, u_old)
    got = stokes.solve(f, n, L, alpha, mu, u_old)
    assert np.max(np.abs(got - want)) < 1e-10 * max(1.0, np.max(np.abs(want)))


def test_stencil_helpers_match_dense_blocks():
    """oracle.stokes.div / grad / lap are the D, G and L blocks of the node-by-node assembly."""
    n, L = (5, 3, 4), (1.0, 0.6, 1.7)
    dim, N = 3, 60
    A = _dense_system(n, L, 0.0, 1.0)
    rng = np.random.default_rng(3)
    u = _field(rng, n)
    p = rng.standard_normal(tuple(reversed(n)))
    uf = np.concatenate([u[a].ravel() for a in range(dim)])
    assert np.allclose(stokes.div(u, n, L).ravel(), A[dim * N:, :dim * N] @ uf, atol=1e-12)
    G = A[:dim * N, dim * N:]
    assert np.allclose(np.concatenate([g.ravel() for g in stokes.grad(p, n, L)]), G @ p.ravel(), atol=1e-12)
    assert np.allclose(np.concatenate([g.ravel() for g in stokes.lap(u, n, L)]), -(A[:dim * N, :dim * N] @ uf),
                       atol=1e-10)
    assert np.allclose(G, -A[dim * N:, :dim * N].T)            # G = -D^T


@pytest.mark.parametrize("m", [1, 2])
def test_stokes_shear_wave_closed_form(m):
    """f = (sin(2 pi m y / L_y), 0, 0) is divergence-free; u = f / (alpha + mu (2 sin(pi m / n_y) / h_y)^2)."""
    n, L, alpha, mu = (8, 6, 5), (1.0, 1.5, 0.75), 4.0, 0.3
    hy = L[1] / n[1]
    y = (np.arange(n[1]) + 0.5) * hy                         # component x sits at cell-centre height in y
    f = np.zeros((3,) + tuple(reversed(n)))
    f[0] = np.sin(2 * np.pi * m * y / L[1])[None, :, None]
    lam = (2.0 * np.sin(np.pi * m / n[1]) / hy) ** 2
    u = stokes.solve(f, n, L, alpha, mu)
    assert np.max(np.abs(u[0] - f[0] / (alpha + mu * lam))) < 1e-13
    assert np.max(np.abs(u[1:])) < 1e-13


def test_stokes_gradient_force_makes_no_flow():
    """f = G phi is balanced by the pressure p = phi: u = 0."""
    n, L = (6, 5, 4), (1.0, 0.8, 1.2)
    h = [L[b] / n[b] for b in range(3)]
    rng = np.random.default_rng(11)
    phi = rng.standard_normal(tuple(reversed(n)))
    f = np.zeros((3,) + tuple(reversed(n)))
    for idx in _nodes(n):                                    # node by node, independent of oracle.stokes.grad
        x, y, z = idx
        for a in range(3):
            dn = list(idx); dn[a] -= 1
            f[a, z, y, x] = (phi[z, y, x] - phi[dn[2] % n[2], dn[1] % n[1], dn[0] % n[0]]) / h[a]
    u = stokes.solve(f, n, L, 2.5, 0.4)
    assert np.max(np.abs(u)) < 1e-12 * np.max(np.abs(f))


def test_stokes_residuals_on_a_larger_grid():
    """D u = 0 and alpha u - mu L u - g is a discrete gradient (its discrete curl vanishes)."""
    n, L, alpha, mu = (16, 12, 10), (1.0, 0.75, 0.625), 1.0, 0.05
    rng = np.random.default_rng(5)
    f, u_old = _field(rng, n), _field(rng, n)
    u = stokes.solve(f, n, L, alpha, mu, u_old)
    scale = np.max(np.abs(u)) / min(L[b] / n[b] for b in range(3))
    assert np.max(np.abs(stokes.div(u, n, L))) < 1e-12 * scale
    r = alpha * u - mu * stokes.lap(u, n, L) - (alpha * u_old + f)   # = -G p
    h = [L[b] / n[b] for b in range(3)]
    for a, b in [(0, 1), (1, 2), (0, 2)]:
        # (r_b[i] - r_b[i - e_a]) / h_a - (r_a[i] - r_a[i - e_b]) / h_b = 0 for r = G p
        ax_a, ax_b = 2 - a, 2 - b
        curl = (r[b] - np.roll(r[b], 1, axis=ax_a)) / h[a] - (r[a] - np.roll(r[a], 1, axis=ax_b)) / h[b]
        assert np.max(np.abs(curl)) < 1e-9 * np.max(np.abs(r)) / min(h)


def test_stokes_mean_mode():
    n, L = (4, 6), (1.0, 1.0)
    f = np.full((2, 6, 4), 0.75)
    f[1] = -1.0
    u = stokes.solve(f, n, L, 2.0, 1.0)
    assert np.allclose(u[0], 0.375) and np.allclose(u[1], -0.5)
    assert np.max(np.abs(stokes.solve(f, n, L, 0.0, 1.0))) < 1e-14


@pytest.mark.parametrize("mutation", [1, 2, 3, 4])
def test_stokes_mutations_caught(mutation):
    n, L, alpha, mu, _ = CASES[2]
    rng = np.random.default_rng(1)
    f, u_old = _field(rng, n), _field(rng, n)
    want = _brute(f, n, L, alpha, mu, u_old)
    stokes.set_mutation(mutation)
    try:
        got = stokes.solve(f, n, L, alpha, mu, u_old)
    finally:
        stokes.set_mutation(0)
    assert np.max(np.abs(got - want)) > 1e-3
