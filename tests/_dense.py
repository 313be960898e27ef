"""Dense brute-force spreading matrix, a code path independent of the oracle.

S[k, j] = h^-d prod_b phi((x_k - X_j)_b / h_b), summed over every periodic
image of X_j: the regularised delta of Section 2 on a periodic box, written
with no cell map, no shifts and no floor.  Used only to pin the oracle on
tiny grids.  phi is typed here a second time from the kernel formulas of
Peskin (2002) and Roma, Peskin and Berger (1999) in their original forms, and
the 6-point B-spline by the Cox-de Boor recursion (not the piecewise
polynomial the oracle uses); the closed-form pins in test_oracle_pins.py pin
both copies.
"""
import itertools

import numpy as np


def phi_std(r):
    a = np.abs(r)
    inner = (3 - 2 * a + np.sqrt(np.clip(1 + 4 * a - 4 * a * a, 0, None))) / 8
    outer = (5 - 2 * a - np.sqrt(np.clip(-7 + 12 * a - 4 * a * a, 0, None))) / 8
    return np.where(a <= 1, inner, np.where(a < 2, outer, 0.0))


def phi_cos(r):
    return np.where(np.abs(r) < 2, 0.25 * (1 + np.cos(np.pi * r / 2)), 0.0)


def phi_roma3(r):
    a = np.abs(r)
    inner = (1 + np.sqrt(np.clip(1 - 3 * a * a, 0, None))) / 3
    outer = (5 - 3 * a - np.sqrt(np.clip(1 - 3 * (1 - a) ** 2, 0, None))) / 6
    return np.where(a <= 0.5, inner, np.where(a < 1.5, outer, 0.0))


def bspline(p, x):
    """Cardinal B-spline of degree p on [0, p + 1] by the Cox-de Boor recursion."""
    x = np.asarray(x, dtype=np.float64)
    if p == 0:
        return np.where((x >= 0) & (x < 1), 1.0, 0.0)
    return (x * bspline(p - 1, x) + (p + 1 - x) * bspline(p - 1, x - 1)) / p


def phi_bspline6(r):
    return bspline(5, np.asarray(r, dtype=np.float64) + 3.0)


PHI = {0: phi_std, 1: phi_cos, 2: phi_roma3, 3: phi_bspline6}


def node_positions(n, L, xi):
    """Positions h (i + xi) of every node, x fastest, shape (ncell, d)."""
    d = len(n)
    axes = [L[b] / n[b] * (np.arange(n[b]) + xi[b]) for b in range(d)]
    mesh = np.meshgrid(*reversed(axes), indexing="ij")       # z, y, x order
    return np.stack([m.ravel() for m in reversed(mesh)], axis=1)


def dense_S(n, L, xi, kernel, X, bounded=()):
    """bounded[b] True: dimension b is not periodic (no images along it)."""
    d = len(n)
    h = np.array([L[b] / n[b] for b in range(d)])
    phi = PHI[kernel]
    xk = node_positions(n, L, xi)
    S = np.zeros((len(xk), len(X)))
    lo = int(np.floor(np.min(X / np.array(L[:d])))) - 3 if len(X) else -3
    hi = int(np.ceil(np.max(X / np.array(L[:d])))) + 3 if len(X) else 3
    span = [range(0, 1) if (b < len(bounded) and bounded[b]) else range(-hi, -lo + 1) for b in range(d)]
    for img in itertools.product(*span):
        shift = np.array(img) * np.array(L[:d])
        diff = (xk[:, None, :] - (X[None, :, :] + shift)) / h
        S += np.prod(phi(diff), axis=2)
    return S / np.prod(h)
