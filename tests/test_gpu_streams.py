"""Several timesteps streamed through the C ABI with host buffers, as the
end-to-end benchmark runs them: positions and forces uploaded on one stream,
U, the new positions and f downloaded on another, the kernels on a third,
ordered by events only, so a step's downloads overlap the next step's
kernels.  The host results must equal, bit for bit, the same steps issued
one call after another on one stream (every sum has a fixed order, so any
copy or kernel that ran out of order shows up as a difference)."""
import numpy as np
import pytest
import torch

import ib_inputs
from _gpu import dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    from paper_2012_06646_gb300 import build
    build()
    from paper_2012_06646_gb300.plan import Plan
    return Plan


def test_streamed_steps_equal_sequential_steps(P):
    n, L, npts, nsteps, dt = (48, 40, 56), (1.0, 0.8, 1.1), 60_000, 5, 0.02
    X0 = ib_inputs.uniform_points(71, npts, L, 3)
    Gh = [torch.from_numpy(ib_inputs.normal_array(72 + k, (npts, 3))).pin_memory() for k in range(3)]
    us = [dev(ib_inputs.normal_array(80 + k, (3, 56, 40, 48))) for k in range(2)]
    plan = P(3, n, L, max_points=npts)

    # one call after another on the current stream
    Xc = dev(X0)
    Gc = torch.empty((npts, 3), dtype=torch.float32, device="cuda")
    for s in range(nsteps):
        Gc.copy_(Gh[s % len(Gh)])
        plan.bin(Xc)
        Uc = plan.interpolate(Xc, us[s % len(us)], reuse_bins=True)
        Xnc = plan.advect(Xc, Uc, dt)
        fc = plan.spread(Xc, Gc, reuse_bins=True)
        Xc = Xnc
    torch.cuda.synchronize()
    X_ref, U_ref, f_ref = Xc.cpu(), Uc.cpu(), fc.cpu()

    # streamed: uploads, kernels and downloads on three streams, ordered by events
    Xh = torch.from_numpy(X0).pin_memory()
    Uh = torch.empty((npts, 3), dtype=torch.float32).pin_memory()
    fh = torch.empty(plan.grid_shape(), dtype=torch.float32).pin_memory()
    Xds = [torch.empty((npts, 3), dtype=torch.float32, device="cuda") for _ in range(2)]
    Xn = torch.empty_like(Xds[0])
    U = torch.empty_like(Xds[0])
    Gd = torch.empty_like(Xds[0])
    f = torch.empty(plan.grid_shape(), dtype=torch.float32, device="cuda")
    st, up, dn = torch.cuda.Stream(), torch.cuda.Stream(), torch.cuda.Stream()
    st.wait_stream(torch.cuda.current_stream())
    prev, prev2_sp = None, None
    for s in range(nsteps):
        xdb = Xds[s % 2]
        if prev is not None:
            up.wait_event(prev["xdown"])       # the host copy of X is the previous step's result
        else:
            up.wait_stream(st)
        if prev2_sp is not None:
            up.wait_event(prev2_sp)
        with torch.cuda.stream(up):
            xdb.copy_(Xh, non_blocking=True)
        e_xup = torch.cuda.Event()
        e_xup.record(up)
        if prev is not None:
            up.wait_event(prev["sp"])
        with torch.cuda.stream(up):
            Gd.copy_(Gh[s % len(Gh)], non_blocking=True)
        e_g = torch.cuda.Event()
        e_g.record(up)
        st.wait_event(e_xup)
        plan.bin(xdb, stream=st)
        if prev is not None:
            st.wait_event(prev["udown"])
        plan.interpolate(xdb, us[s % len(us)], U=U, reuse_bins=True, stream=st)
        plan.advect(xdb, U, dt, out=Xn, stream=st)
        e_ad = torch.cuda.Event()
        e_ad.record(st)
        dn.wait_event(e_ad)
        with torch.cuda.stream(dn):
            Xh.copy_(Xn, non_blocking=True)
        e_xd = torch.cuda.Event()
        e_xd.record(dn)
        with torch.cuda.stream(dn):
            Uh.copy_(U, non_blocking=True)
        e_ud = torch.cuda.Event()
        e_ud.record(dn)
        st.wait_event(e_g)
        if prev is not None:
            st.wait_event(prev["fdown"])
        plan.spread(xdb, Gd, f=f, reuse_bins=True, stream=st)
        e_sp = torch.cuda.Event()
        e_sp.record(st)
        dn.wait_event(e_sp)
        with torch.cuda.stream(dn):
            fh.copy_(f, non_blocking=True)
        e_fd = torch.cuda.Event()
        e_fd.record(dn)
        prev2_sp = prev["sp"] if prev is not None else None
        prev = {"xdown": e_xd, "udown": e_ud, "fdown": e_fd, "sp": e_sp}
    st.wait_stream(up)
    st.wait_stream(dn)
    st.synchronize()
    plan.check(st)
    assert torch.equal(Xh, X_ref)
    assert torch.equal(Uh, U_ref)
    assert torch.equal(fh, f_ref)
    assert np.isfinite(fh.numpy()).all()
