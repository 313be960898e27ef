"""Served batch: each job's result is the same alone and in a mix; waves of uneven
jobs match the oracle; the continuous-batching loop completes every request."""
import numpy as np
import pytest
import torch

import ib_inputs
from _gpu import assert_interp_close, assert_spread_close, dev, host

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mods():
    from paper_2012_06646_gb300 import build
    build()
    from paper_2012_06646_gb300 import serve
    from paper_2012_06646_gb300.plan import Batch, Plan
    return Plan, Batch, serve


def _jobs(seed, count, grids=(8, 17, 32, 48), n_lo=50, n_hi=3000):
    return ib_inputs.job_mix(seed, count, grids=grids, n_lo=n_lo, n_hi=n_hi)


def test_batched_wave_equals_single_jobs_and_oracle(mods, orc):
    Plan, Batch, serve = mods
    specs = _jobs(5, 12)
    batch = Batch(dim=3, max_jobs=16, max_points=1 << 16, max_cells=1 << 20)
    jobs, bufs = [], []
    for sp in specs:
        X = ib_inputs.job_points(sp)
        G = ib_inputs.normal_array(sp.seed, (sp.npts, 3), purpose="job-G")
        Xd, Gd = dev(X), dev(G)
        f = torch.empty((3, sp.N, sp.N, sp.N), device="cuda")
        U = torch.empty_like(Xd)
        bufs.append((X, G, Xd, Gd, f, U))
        jobs.append(batch.job_struct((sp.N,) * 3, (1.0,) * 3, Xd, G=Gd, f=f, u=f, U=U))
    batch.run(jobs)
    batch.check()
    for sp, (X, G, Xd, Gd, f, U) in zip(specs, bufs):
        plan = Plan(3, (sp.N,) * 3, (1.0,) * 3, max_points=sp.npts)
        f1 = plan.spread(Xd, Gd)
        U1 = plan.interpolate(Xd, f1, reuse_bins=True)
        # identical alone and in the mix (same bins, tiles and summation order per job)
        assert torch.equal(f, f1) and torch.equal(U, U1)
        g = orc.Grid(dim=3, n=(sp.N,) * 3, L=(1.0,) * 3)
        f_ref, fabs = orc.spread(g, X, G)
        assert_spread_close(host(f), f_ref, fabs)
        U_ref, Uabs = orc.interp(g, X, host(f).astype(np.float64))
        assert_interp_close(host(U), U_ref, Uabs)
        plan.close()
    # a wave of one job runs the single-job launches: the same result as in the mix
    for sp, (X, G, Xd, Gd, f, U) in list(zip(specs, bufs))[:3]:
        f2 = torch.empty_like(f)
        U2 = torch.empty_like(U)
        batch.run([batch.job_struct((sp.N,) * 3, (1.0,) * 3, Xd, G=Gd, f=f2, u=f2, U=U2)])
        batch.check()
        assert torch.equal(f2, f) and torch.equal(U2, U)


def test_batch_run_host_equals_device_batch(mods):
    Plan, Batch, serve = mods
    specs = _jobs(7, 10)
    dbatch = Batch(dim=3, max_jobs=16, max_points=1 << 16, max_cells=1 << 20)
    hbatch = Batch(dim=3, max_jobs=16, max_points=1 << 16, max_cells=1 << 20, host_io=True)
    jobs, outs, hjobs, keep = [], [], [], []
    for sp in specs:
        X = ib_inputs.job_points(sp)
        G = ib_inputs.normal_array(sp.seed, (sp.npts, 3), purpose="job-G")
        Xd, Gd = dev(X), dev(G)
        f = torch.empty((3, sp.N, sp.N, sp.N), device="cuda")
        U = torch.empty_like(Xd)
        keep.append((Xd, Gd, f))             # the device batch reads them when it runs
        outs.append(U)
        jobs.append(dbatch.job_struct((sp.N,) * 3, (1.0,) * 3, Xd, G=Gd, f=f, u=f, U=U))
        Uh = torch.full((sp.npts, 3), float("nan")).pin_memory()
        hjobs.append(((sp.N,) * 3, (1.0,) * 3, torch.from_numpy(X).pin_memory(), torch.from_numpy(G).pin_memory(), Uh))
    dbatch.run(jobs)
    hbatch.run_host(hjobs)
    torch.cuda.synchronize()
    dbatch.check()
    hbatch.check()
    for U, (_, _, _, _, Uh) in zip(outs, hjobs):
        assert torch.equal(U.cpu(), Uh)
    # two waves in a row on the same batch object reuse its buffers
    hbatch.run_host(hjobs[:3])
    torch.cuda.synchronize()
    for U, (_, _, _, _, Uh) in zip(outs[:3], hjobs[:3]):
        assert torch.equal(U.cpu(), Uh)
    dbatch.close()
    hbatch.close()


def test_wave_status_reports_each_host_wave_without_a_sync(mods):
    """ib_batch_wave_status: the error word as the last host-I/O wave left it, read from
    pinned memory that the wave's stream wrote; ib_batch_check still reads and clears it."""
    from paper_2012_06646_gb300 import _abi
    Plan, Batch, serve = mods
    b = Batch(dim=3, max_jobs=4, max_points=1 << 16, max_cells=1 << 20, host_io=True)
    specs = _jobs(11, 3)
    waves = []
    for bad in (False, True, False):
        jobs = []
        for sp in specs:
            X = ib_inputs.job_points(sp)
            if bad:
                X[sp.npts // 2] = np.nan
            G = ib_inputs.normal_array(sp.seed, (sp.npts, 3), purpose="job-G")
            jobs.append(((sp.N,) * 3, (1.0,) * 3, torch.from_numpy(X).pin_memory(), torch.from_numpy(G).pin_memory(),
                         torch.empty((sp.npts, 3)).pin_memory()))
        waves.append(jobs)
    s = torch.cuda.current_stream()
    b.run_host(waves[0], stream=s)
    s.synchronize()
    assert b.wave_status() == _abi.IB_OK
    b.run_host(waves[1], stream=s)
    s.synchronize()
    assert b.wave_status() == _abi.IB_ERR_NONFINITE
    assert b.status(s) == _abi.IB_ERR_NONFINITE              # read and cleared
    b.run_host(waves[2], stream=s)
    s.synchronize()
    assert b.wave_status() == _abi.IB_OK
    assert all(bool(torch.isnan(U[sp.npts // 2]).all()) for (_, _, _, _, U), sp in zip(waves[1], specs))
    b.close()


def test_server_continuous_batching_matches_single_loop(mods):
    Plan, Batch, serve = mods
    specs = _jobs(9, 60)
    arrivals = ib_inputs.poisson_arrivals(9, len(specs), rate_per_s=4000.0)
    reqs = serve.make_requests(specs, arrivals=arrivals)
    srv = serve.Server(nstreams=3, max_jobs=16, max_points=1 << 16, max_cells=1 << 19)
    st = srv.serve(reqs)
    assert st.jobs == len(reqs) and all(r.t_done >= r.arrival for r in reqs)
    assert st.waves >= 2
    mixed = [r.U.clone() for r in reqs]
    reqs2 = serve.make_requests(specs, arrivals=arrivals)
    st2 = serve.single_job_loop(reqs2)
    assert st2.jobs == len(reqs2)
    for a, r in zip(mixed, reqs2):
        assert torch.equal(a, r.U)
    srv.close()


def test_server_admission_respects_budget(mods):
    Plan, Batch, serve = mods
    specs = _jobs(11, 20, grids=(32,), n_lo=1000, n_hi=1001)
    reqs = serve.make_requests(specs)
    srv = serve.Server(nstreams=2, max_jobs=8, max_points=1 << 16, max_cells=1 << 18)
    one = srv.footprint(reqs[0])[0]
    srv.budget = int(2.5 * one)                  # at most two jobs in flight
    st = srv.serve(reqs, realtime=False)
    assert st.jobs == 20
    assert st.max_inflight_bytes <= srv.budget
    srv.close()
