"""The full IB timestep (Section 2, steps (a)-(g)) on the GPU through the C
ABI (paper_2012_06646_gb300.step.IBStep: bin, interpolate, advect, spread,
Stokes solve, interpolate, advect), against the same loop written with the
FP64 oracles (oracle.interp / oracle.spread and oracle.stokes.solve), with
the same tether forces of step (c) on both sides.

Tolerances: FP64, three steps: positions within 1e-11 L and velocities within
1e-10 max|u| (each call is exact to rounding; three steps add a few rounding
levels).  FP32, one step: positions within 2.4e-7 L (two roundings of a
position below 1, whose FP32 spacing is 6e-8, in steps (b) and (g)) plus
5e-5 of the step's largest displacement (k times a velocity carrying the
errors below), and velocities within 5e-5 max|u| (the spread, the solve and
the input rounding each contribute about 1e-5 of the field's scale).
"""
import numpy as np
import pytest
import torch

import ib_inputs
from _gpu import dev, host
from oracle import stokes

pytestmark = pytest.mark.gpu

KAPPA = 1.0


def tether_np(Xs, X0, L):
    d = X0 - Xs
    d -= L * np.round(d / L)
    return KAPPA * d


def tether_torch(Xs, X0, L):
    d = X0 - Xs
    d = d - L * torch.round(d / L)
    return (KAPPA * d).contiguous()


def oracle_loop(orc, n, L, X, u, X0, rho, mu, k, steps):
    g = orc.Grid(len(n), n, L, mac=True)
    Lv = np.asarray(L, dtype=np.float64)
    X = X.astype(np.float64)
    u = u.astype(np.float64)
    for _ in range(steps):
        U, _ = orc.interp(g, X, u)                                   # (a)
        Xs = np.mod(X + k * U, Lv)                                   # (b)
        G = tether_np(Xs, X0, Lv)                                    # (c)
        f, _ = orc.spread(g, Xs, G)                                  # (d)
        u = stokes.solve(f, n, L, rho / k, mu, u)                    # (e)
        U, _ = orc.interp(g, X, u)                                   # (f)
        X = np.mod(X + k * U, Lv)                                    # (g)
    return X, u


def periodic_err(a, b, L):
    d = np.abs(a - b)
    return np.minimum(d, np.asarray(L) - d)


@pytest.mark.parametrize("dtype,steps", [(np.float64, 3), (np.float32, 1)])
def test_ib_step_matches_oracle_loop(orc, dtype, steps):
    from paper_2012_06646_gb300 import build
    build()
    from paper_2012_06646_gb300.step import IBStep
    n, L = (24, 20, 16), (1.0, 1.0, 0.8)
    rho, mu, k = 1.0, 0.05, 0.01
    npts = 600
    X = ib_inputs.uniform_points(41, npts, L, 3, dtype=dtype)
    # tether anchors about 0.01 from the points: forces of order 0.01 per point
    X0 = np.mod(X.astype(np.float64) + 0.01 * ib_inputs.normal_array(42, (npts, 3), dtype=np.float64),
                np.asarray(L))
    u = (0.1 * ib_inputs.normal_array(43, (3,) + tuple(reversed(n)), dtype=np.float64, purpose="u")).astype(dtype)
    tdt = torch.float64 if dtype == np.float64 else torch.float32
    stepper = IBStep(3, n, L, rho, mu, k, dtype=tdt, max_points=npts)
    Xd, ud = dev(X), dev(u)
    X0d = dev(X0).to(tdt)
    Lt = torch.tensor(L, dtype=tdt, device="cuda")
    for _ in range(steps):
        Xd, ud = stepper.step(Xd, ud, lambda Xs: tether_torch(Xs, X0d, Lt))
    stepper.plan_n.check()
    Xw, uw = oracle_loop(orc, n, L, X, u, X0, rho, mu, k, steps)
    Xg, ug = host(Xd).astype(np.float64), host(ud).astype(np.float64)
    disp = periodic_err(Xw, X.astype(np.float64), L).max()
    if dtype == np.float64:
        xtol, utol = 1e-11 * max(L), 1e-10
    else:
        xtol, utol = 2.4e-7 * max(L) + 5e-5 * disp, 5e-5
    assert periodic_err(Xg, Xw, L).max() <= xtol
    assert np.abs(ug - uw).max() <= utol * np.abs(uw).max()
    assert disp > 100 * xtol                 # the points moved by much more than the tolerance
    stepper.close()


def test_ib_step_2d_matches_oracle_loop(orc):
    """The same loop in 2-D (MAC grid, FP64, three steps)."""
    from paper_2012_06646_gb300 import build
    build()
    from paper_2012_06646_gb300.step import IBStep
    n, L = (40, 24), (1.0, 0.6)
    rho, mu, k, npts, steps = 1.0, 0.02, 0.01, 300, 3
    X = ib_inputs.uniform_points(71, npts, L, 2, dtype=np.float64)
    X0 = np.mod(X + 0.01 * ib_inputs.normal_array(72, (npts, 2), dtype=np.float64), np.asarray(L))
    u = 0.1 * ib_inputs.normal_array(73, (2, 24, 40), dtype=np.float64, purpose="u")
    stepper = IBStep(2, n, L, rho, mu, k, dtype=torch.float64, max_points=npts)
    Xd, ud = dev(X), dev(u)
    X0d = dev(X0)
    Lt = torch.tensor(L, dtype=torch.float64, device="cuda")
    for _ in range(steps):
        Xd, ud = stepper.step(Xd, ud, lambda Xs: tether_torch(Xs, X0d, Lt))
    stepper.plan_n.check()
    Xw, uw = oracle_loop(orc, n, L, X, u, X0, rho, mu, k, steps)
    assert periodic_err(host(Xd), Xw, L).max() <= 1e-11
    assert np.abs(host(ud) - uw).max() <= 1e-10 * np.abs(uw).max()
    stepper.close()
