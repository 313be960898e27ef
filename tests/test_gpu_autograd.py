"""Differentiation: autograd through the CUDA kernels against the oracle gradient
and FP64 central finite differences (spread with interpolation backward and the
delta-derivative position gradient)."""
import numpy as np
import pytest
import torch

import ib_inputs
from _gpu import FLOOR32, assert_interp_close, dev, host

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mods():
    from paper_2012_06646_gb300 import build
    build()
    from paper_2012_06646_gb300 import autograd
    from paper_2012_06646_gb300.plan import Plan
    return Plan, autograd


def test_spread_gradients_128_mac_2e5(mods, orc):
    """128^3 MAC grid, 2x10^5 points, loss = sum(w * spread(G, X)), w ~ N(0,1)."""
    Plan, ag = mods
    n, npts = (128, 128, 128), 200_000
    plan = Plan(3, n, (1.0, 1.0, 1.0), max_points=npts)
    X = ib_inputs.uniform_points(51, npts, (1.0, 1.0, 1.0), 3)
    G = ib_inputs.normal_array(52, (npts, 3))
    w = ib_inputs.normal_array(53, plan.grid_shape())
    Xd = dev(X).requires_grad_(True)
    Gd = dev(G).requires_grad_(True)
    loss = (dev(w) * ag.spread(Xd, Gd, plan)).sum()
    gX, gG = torch.autograd.grad(loss, (Xd, Gd))
    g = orc.Grid(dim=3, n=n, L=(1.0, 1.0, 1.0))
    hmd = orc.inv_cell_volume(g)
    Uw, Uwabs = orc.interp(g, X, w)
    assert_interp_close(host(gG), hmd * Uw, hmd * Uwabs, what="dL/dG")
    D, Dabs = orc.pos_grad(g, X, w, G)
    assert_interp_close(host(gX), hmd * D, hmd * Dabs, rel=2e-5, what="dL/dX")


def test_interpolation_gradients(mods, orc):
    Plan, ag = mods
    n, npts = (40, 32, 24), 5000
    plan = Plan(3, n, (1.0, 0.8, 0.6), max_points=npts)
    g = orc.Grid(dim=3, n=n, L=(1.0, 0.8, 0.6))
    X = ib_inputs.uniform_points(61, npts, g.L, 3)
    u = ib_inputs.normal_array(62, plan.grid_shape())
    v = ib_inputs.normal_array(63, (npts, 3))
    Xd = dev(X).requires_grad_(True)
    ud = dev(u).requires_grad_(True)
    loss = (dev(v) * ag.interpolate(Xd, ud, plan)).sum()
    gX, gu = torch.autograd.grad(loss, (Xd, ud))
    hmd = orc.inv_cell_volume(g)
    f, fabs = orc.spread(g, X, v)          # h^-d W^T v
    from _gpu import assert_spread_close
    assert_spread_close(host(gu), f / hmd, fabs / hmd, what="dL/du")
    D, Dabs = orc.pos_grad(g, X, u, v)
    assert_interp_close(host(gX), D, Dabs, rel=2e-5, what="dL/dX")


def test_fd_16cubed_200_points_fp64(mods, orc):
    """FP64 plan: autograd gradient against central differences (eps = 1e-6) of the oracle loss."""
    Plan, ag = mods
    n = (16, 16, 16)
    plan = Plan(3, n, (1.0, 1.0, 1.0), dtype=torch.float64, max_points=200)
    g = orc.Grid(dim=3, n=n, L=(1.0, 1.0, 1.0))
    X = ib_inputs.uniform_points(71, 200, g.L, 3, dtype=np.float64)
    G = ib_inputs.normal_array(72, (200, 3), dtype=np.float64)
    w = ib_inputs.normal_array(73, plan.grid_shape(), dtype=np.float64)
    Xd = dev(X).requires_grad_(True)
    Gd = dev(G).requires_grad_(True)
    loss = (dev(w) * ag.spread(Xd, Gd, plan)).sum()
    gX, gG = torch.autograd.grad(loss, (Xd, Gd))
    gX = host(gX)
    eps = 1e-6
    fd = np.zeros_like(X)
    for j in range(0, 200, 10):
        for b in range(3):
            Xp, Xm = X.copy(), X.copy()
            Xp[j, b] += eps
            Xm[j, b] -= eps
            fd[j, b] = (np.sum(w * orc.spread(g, Xp, G)[0]) - np.sum(w * orc.spread(g, Xm, G)[0])) / (2 * eps)
    sel = np.arange(0, 200, 10)
    assert np.max(np.abs(gX[sel] - fd[sel])) <= 1e-6 * np.max(np.abs(gX))
    hmd = orc.inv_cell_volume(g)
    D, _ = orc.pos_grad(g, X, w, G)
    assert np.max(np.abs(gX - hmd * D)) <= 1e-12 * np.max(np.abs(hmd * D))
    Uw, _ = orc.interp(g, X, w)
    assert np.max(np.abs(host(gG) - hmd * Uw)) <= 1e-12 * np.max(np.abs(hmd * Uw))


def test_gradcheck_fp64(mods):
    Plan, ag = mods
    plan = Plan(3, (8, 8, 8), (1.0, 1.0, 1.0), dtype=torch.float64, max_points=12)
    X = dev(ib_inputs.uniform_points(81, 12, (1.0, 1.0, 1.0), 3, dtype=np.float64)).requires_grad_(True)
    G = dev(ib_inputs.normal_array(82, (12, 3), dtype=np.float64)).requires_grad_(True)
    u = dev(ib_inputs.normal_array(83, plan.grid_shape(), dtype=np.float64)).requires_grad_(True)
    assert torch.autograd.gradcheck(lambda x, gg: ag.spread(x, gg, plan), (X, G), eps=1e-6, atol=1e-5, rtol=1e-4)
    assert torch.autograd.gradcheck(lambda x, uu: ag.interpolate(x, uu, plan), (X, u), eps=1e-6, atol=1e-5, rtol=1e-4)


def test_backward_rebins_after_other_calls(mods, orc):
    """The backward reuses the forward's bins only while the plan holds them: here the plan
    interpolates other points between forward and backward, so the backward must bin X again."""
    Plan, ag = mods
    n, npts = (16, 16, 16), 300
    plan = Plan(3, n, (1.0, 1.0, 1.0), max_points=npts)
    X = ib_inputs.uniform_points(81, npts, (1.0, 1.0, 1.0), 3)
    G = ib_inputs.normal_array(82, (npts, 3))
    w = ib_inputs.normal_array(83, plan.grid_shape())
    Xd = dev(X).requires_grad_(True)
    Gd = dev(G).requires_grad_(True)
    f = ag.spread(Xd, Gd, plan)
    epoch = plan.bin_epoch
    plan.interpolate(dev(ib_inputs.uniform_points(84, npts, (1.0, 1.0, 1.0), 3)), dev(w))
    assert plan.bin_epoch == epoch + 1
    gX, gG = torch.autograd.grad((dev(w) * f).sum(), (Xd, Gd))
    plan.check()
    g = orc.Grid(dim=3, n=n, L=(1.0, 1.0, 1.0))
    hmd = orc.inv_cell_volume(g)
    Uw, Uwabs = orc.interp(g, X, w)
    assert_interp_close(host(gG), hmd * Uw, hmd * Uwabs, what="dL/dG")
    D, Dabs = orc.pos_grad(g, X, w, G)
    assert_interp_close(host(gX), hmd * D, hmd * Dabs, rel=2e-5, what="dL/dX")
    # and with nothing in between, the bins are reused (no new binning)
    f = ag.spread(Xd, Gd, plan)
    epoch = plan.bin_epoch
    gX2, _ = torch.autograd.grad((dev(w) * f).sum(), (Xd, Gd))
    assert plan.bin_epoch == epoch
    assert torch.equal(gX2, gX)
