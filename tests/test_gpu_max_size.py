"""The largest case the tests run: a 512^3 MAC grid with 2^26 points (half a
point per cell, the benchmark's density).  Cell ids reach 1.3 x 10^8, tile ids
2.6 x 10^5 and spreading-box offsets 1.36 x 10^9 entries, near the top of the
32-bit index ranges the kernels use.  Checked where the oracle can compute it:

  * the bins on every point, by their definition (a permutation sorting the
    cell keys, index order inside a cell, cell starts = counts of smaller keys);
  * spreading and interpolation against the FP64 oracle on two sub-boxes
    (one in the last tiles of the grid), each with the points around it moved
    by a whole number of cells onto a small grid of the same spacing, on which
    no support wraps."""
import numpy as np
import pytest
import torch

import ib_inputs
from _gpu import assert_interp_close, assert_spread_close, dev, host

pytestmark = pytest.mark.gpu

N = 512
NPTS = 1 << 26
R = 20          # sub-box side (nodes)
PAD = 8         # nodes of the small grid on each side of the sub-box
M = R + 2 * PAD


@pytest.fixture(scope="module")
def big():
    from paper_2012_06646_gb300 import build
    build()
    from paper_2012_06646_gb300.plan import Plan
    X = ib_inputs.uniform_points(300, NPTS, (1.0, 1.0, 1.0), 3)
    G = ib_inputs.uniform_array(301, (NPTS, 3))
    u = ib_inputs.wave_field(N)
    plan = Plan(3, (N, N, N), (1.0, 1.0, 1.0), max_points=NPTS)
    Xd, Gd = dev(X), dev(G)
    plan.bin(Xd)
    f = plan.spread(Xd, Gd, reuse_bins=True)
    ud = dev(u)
    U = plan.interpolate(Xd, ud, reuse_bins=True)
    plan.check()
    yield plan, X, G, u, Xd, f, U
    plan.close()


def test_bins_at_512_cubed(big):
    plan, X, G, u, Xd, f, U = big
    perm, start = plan.bins()
    c = torch.floor(Xd.double() * N).long()             # cells of xi = 0 (N / L = 512 exactly)
    key = c[:, 0] + N * (c[:, 1] + N * c[:, 2])
    assert int(torch.bincount(perm, minlength=NPTS).max()) == 1     # a permutation
    ks = key[perm]
    assert bool((ks[1:] >= ks[:-1]).all())
    tie = ks[1:] == ks[:-1]
    assert bool((perm[1:][tie] > perm[:-1][tie]).all())              # index order inside a cell
    counts = torch.bincount(key, minlength=N ** 3)
    ref = torch.zeros(N ** 3 + 1, dtype=torch.int64, device=key.device)
    ref[1:] = torch.cumsum(counts, 0)
    assert torch.equal(start[: N ** 3 + 1], ref)


@pytest.mark.parametrize("r0", [200, N - R - PAD])
def test_spread_and_interp_on_sub_boxes(big, orc, r0):
    plan, X, G, u, Xd, f, U = big
    s = r0 - PAD                                          # small-grid node 0 = grid node s
    x512 = X.astype(np.float64) * N
    near = np.all((x512 >= r0 - 4) & (x512 < r0 + R + 4), axis=1)
    idx = np.nonzero(near)[0]
    Xs = X[idx].astype(np.float64) - s / N                # exact in FP64: whole cells of 1/512
    g = orc.Grid(dim=3, n=(M, M, M), L=(M / N,) * 3, mac=True)
    f_ref, fabs = orc.spread(g, Xs, G[idx])
    sl = slice(PAD, PAD + R)
    fg = host(f[:, r0:r0 + R, r0:r0 + R, r0:r0 + R])
    assert_spread_close(fg, f_ref[:, sl, sl, sl], fabs[:, sl, sl, sl], what=f"spread, sub-box at {r0}")
    inner = np.all((x512[idx] >= r0) & (x512[idx] < r0 + R), axis=1)
    pts = idx[inner]
    assert len(pts) > 1000
    ub = u[:, s:s + M, s:s + M, s:s + M].astype(np.float64)
    U_ref, Uabs = orc.interp(g, X[pts].astype(np.float64) - s / N, ub)
    assert_interp_close(host(U[torch.from_numpy(pts).cuda()]), U_ref, Uabs, what=f"interp, sub-box at {r0}")
