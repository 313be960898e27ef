"""One immersed-boundary timestep (Section 2, steps (a)-(g)) on a periodic MAC grid.

Marshalling only: every step runs in libibgb.so through its C entry points.
The Lagrangian forces of step (c) come from the caller (`forces(X*)` returns
the (npts, dim) array G of F dtheta values; elastic models are outside this
library).  Per step, with timestep k:

  (a) U* = interp(u^n, X^n)                      ib_bin(X^n) + ib_interpolate
  (b) X* = X^n + k U*                            ib_advect
  (c) G* = forces(X*)                            caller
  (d) f* = spread(G*, X*)                        ib_bin(X*) + ib_spread
  (e) u^{n+1}: Stokes solve with f*, u^n         ib_stokes_solve
  (f) U^{n+1} = interp(u^{n+1}, X^n)             ib_interpolate, bins of (a) reused
  (g) X^{n+1} = X^n + k U^{n+1}                  ib_advect

Two plans hold the bins of X^n (used by (a) and (f)) and of X* (used by (d)),
so each step bins twice.  rho_over_k = rho / k of the Stokes solve.
"""

from __future__ import annotations

import torch

from .plan import Plan, Stokes


class IBStep:
    def __init__(self, dim: int, n, L, rho: float, mu: float, k: float, dtype=torch.float32, max_points: int = 0,
                 device=None):
        self.plan_n = Plan(dim, n, L, grid="mac", dtype=dtype, max_points=max_points, device=device)
        self.plan_s = Plan(dim, n, L, grid="mac", dtype=dtype, max_points=max_points, device=device)
        self.fluid = Stokes(dim, n, L, dtype=dtype, device=device)
        self.rho, self.mu, self.k = float(rho), float(mu), float(k)

    def step(self, X, u, forces, X_out=None, u_out=None, stream=None):
        """Returns (X^{n+1}, u^{n+1}); X and u are not modified unless passed as X_out / u_out."""
        pn, ps = self.plan_n, self.plan_s
        pn.bin(X, stream=stream)
        U = pn.interpolate(X, u, reuse_bins=True, stream=stream)                       # (a)
        Xs = pn.advect(X, U, self.k, stream=stream)                                     # (b)
        G = forces(Xs)                                                                  # (c)
        f = ps.spread(Xs, G, stream=stream)                                             # (d)
        u_new = self.fluid.solve(f, u, self.rho / self.k, self.mu, u=u_out, stream=stream)   # (e)
        pn.interpolate(X, u_new, U=U, reuse_bins=True, stream=stream)                   # (f)
        X_new = pn.advect(X, U, self.k, out=X_out, stream=stream)                       # (g)
        return X_new, u_new

    def close(self):
        self.plan_n.close()
        self.plan_s.close()
        self.fluid.close()
