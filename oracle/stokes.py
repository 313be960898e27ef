"""FP64 oracle for the periodic MAC-grid Stokes solve of the IB step (e).

TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
cpu_baseline / reference leg of bench.py may import this module.  It shares
no code with the CUDA library and never imports it.

Grid (Section 2, the MAC grid): cell centres at (i + 1/2) h per dimension;
velocity component a lives at the cell centre shifted by -h e_a / 2, so
component a's node i sits at i h along a and at (j + 1/2) h along the other
dimensions.  Arrays are component-major [a][z][y][x] (x fastest), the layout
of the library's grid fields; numpy axis of dimension b is dim - 1 - b.

Operators (each the plain stencil, periodic wrap):
  div   (D u)[c]      = sum_b (u_b[c + e_b] - u_b[c]) / h_b       (cell centres)
  grad  (G p)_a[i]    = (p[i] - p[i - e_a]) / h_a                 (faces of a)
  lap   (L u)_a[i]    = sum_b (u_a[i + e_b] - 2 u_a[i] + u_a[i - e_b]) / h_b^2

The step (e) in its Stokes limit (the momentum equation of Section 2 with the
convective term dropped, viscous term backward Euler, incompressibility
enforced exactly):  alpha u + G p - mu L u = alpha u_old + f,  D u = 0,
alpha = rho / k.  `solve` takes the discrete Fourier transform of each
component (a library FFT as one step), solves the per-mode 2 x 2 / 3 x 3
system in closed form and transforms back.  With theta_b = 2 pi k_b / n_b the
stencils act on the mode exp(i sum_b theta_b j_b) as
  D_b = (exp(i theta_b) - 1) / h_b,   G_a = -conj(D_a),   L = -sum_b |D_b|^2,
so, writing g = alpha u_old + f and |d|^2 = sum_b |D_b|^2:
  p^ = -(sum_b D_b g^_b) / |d|^2   (apply D to the momentum equation, D u = 0),
  u^_a = (g^_a - G_a p^) / (alpha + mu |d|^2)
       = (g^_a - conj(D_a) (sum_b D_b g^_b) / |d|^2) / (alpha + mu |d|^2),
and at the zero mode u^ = g^ / alpha (0 when alpha = 0).

Pins (tests/test_oracle_stokes.py): a dense least-squares solve of the
real-space saddle-point system assembled cell by cell, the closed-form shear
wave, a gradient force that produces no flow, and the stencil residuals.
"""

from __future__ import annotations

import numpy as np

# Planted-mistake switch for the mutation test (0 = the solve as stated):
# 1 drops the conjugate of D_a, 2 takes the faces at +h/2 (D_b = (1 - exp(-i theta_b)) / h_b),
# 3 drops the projection term, 4 uses h_0 in every dimension.
_mutation = 0


def set_mutation(m: int) -> None:
    global _mutation
    _mutation = int(m)


def _axis(dim: int, b: int) -> int:
    """numpy axis (within one component) of dimension b (x = 0 is the last axis)."""
    return dim - 1 - b


def spacing(n, L):
    return [float(L[b]) / int(n[b]) for b in range(len(n))]


def div(u: np.ndarray, n, L) -> np.ndarray:
    """Cell-centred divergence of the face field u [dim][...]: forward differences."""
    dim = len(n)
    h = spacing(n, L)
    out = np.zeros(u.shape[1:])
    for b in range(dim):
        ax = _axis(dim, b)
        out += (np.roll(u[b], -1, axis=ax) - u[b]) / h[b]
    return out


def grad(p: np.ndarray, n, L) -> np.ndarray:
    """Face gradient of the cell-centred p: backward differences, one component per dimension."""
    dim = len(n)
    h = spacing(n, L)
    return np.stack([(p - np.roll(p, 1, axis=_axis(dim, a))) / h[a] for a in range(dim)])


def lap(u: np.ndarray, n, L) -> np.ndarray:
    """Component-wise 3-point Laplacian of a face field."""
    dim = len(n)
    h = spacing(n, L)
    out = np.zeros_like(u, dtype=np.float64)
    for a in range(u.shape[0]):
        for b in range(dim):
            ax = _axis(dim, b)
            out[a] += (np.roll(u[a], -1, axis=ax) - 2.0 * u[a] + np.roll(u[a], 1, axis=ax)) / h[b] ** 2
    return out


def solve(f, n, L, rho_over_k: float, mu: float, u_old=None) -> np.ndarray:
    """u of the Stokes step (e) for the face force f [dim][...] (FP64)."""
    dim = len(n)
    h = spacing(n, L)
    f = np.asarray(f, dtype=np.float64)
    g = f.copy() if u_old is None else rho_over_k * np.asarray(u_old, dtype=np.float64) + f
    ghat = np.stack([np.fft.fftn(g[a]) for a in range(dim)])
    shape = g.shape[1:]
    # D_b on the mode grid, broadcast along dimension b's axis.
    Dm = []
    for b in range(dim):
        k = np.arange(int(n[b]))
        theta = 2.0 * np.pi * k / int(n[b])
        hb = h[0] if _mutation == 4 else h[b]
        Db = ((1.0 - np.exp(-1j * theta)) if _mutation == 2 else (np.exp(1j * theta) - 1.0)) / hb
        view = [1] * dim
        view[_axis(dim, b)] = int(n[b])
        Dm.append(np.broadcast_to(Db.reshape(view), shape))
    d2 = sum(np.abs(Dm[b]) ** 2 for b in range(dim))
    s = sum(Dm[b] * ghat[b] for b in range(dim))
    zero = d2 == 0.0
    safe = np.where(zero, 1.0, d2)
    uhat = np.empty_like(ghat)
    for a in range(dim):
        proj = 0.0 if _mutation == 3 else (Dm[a] if _mutation == 1 else np.conj(Dm[a])) * s / safe
        ua = (ghat[a] - proj) / (rho_over_k + mu * safe)
        mean = ghat[a] / rho_over_k if rho_over_k > 0.0 else np.zeros_like(ghat[a])
        uhat[a] = np.where(zero, mean, ua)
    return np.stack([np.real(np.fft.ifftn(uhat[a])) for a in range(dim)])
