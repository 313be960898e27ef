"""The served loop's host logic on CPU: the continuous-batching loop of
serve.Server driven by a fake batch object and fake CUDA streams and events
(no GPU), so rejection, cancellation, per-request outcomes and the
degradation to fewer wave slots are checked in the CPU suite too.  The fake
batch 'computes' U = G, or NaN rows for non-finite positions, and reports the
wave's error word the way ib_batch_check does."""
import types

import numpy as np
import pytest
import torch


class FakeEvent:
    def __init__(self, *a, **k):
        self.done = False

    def record(self, stream=None):
        self.done = True

    def query(self):
        return self.done


class FakeStream:
    def __init__(self, *a, **k):
        pass


def make_fake_batch(abi, fail_at=None):
    made = {"n": 0}

    class FakeBatch:
        def __init__(self, dim=3, grid="mac", max_jobs=64, max_points=1 << 22, max_cells=1 << 24,
                     max_tiles=None, host_io=False, device=None, **kw):
            k = made["n"]
            made["n"] += 1
            if fail_at is not None and k >= fail_at:
                raise abi.IBError(abi.IB_ERR_OOM, "ib_batch_create")
            self.desc = types.SimpleNamespace(max_tiles=max_tiles, max_jobs=max_jobs, max_points=max_points)
            self.err = abi.IB_OK
            self.waves = []

        def job_struct(self, n, L, X, **kw):
            return types.SimpleNamespace(n=n, npts=int(X.shape[0]))

        def job_footprint(self, job):
            if min(job.n) < 1:
                raise abi.IBError(abi.IB_ERR_INVALID_ARG, "ib_batch_job_footprint")
            tiles = int(np.prod([(v + 7) // 8 for v in job.n]))
            return 36 * job.npts + 12 * int(np.prod(job.n)), tiles

        def run_host(self, jobs, stream=None):
            self.waves.append(len(jobs))
            for n, L, X, G, U in jobs:
                bad = ~torch.isfinite(X).all(dim=1)
                U.copy_(G)
                U[bad] = float("nan")
                if bool(bad.any()):
                    self.err = abi.IB_ERR_NONFINITE

        def status(self, stream=None):
            e, self.err = self.err, abi.IB_OK
            return e

        def wave_status(self):
            return self.err                    # the word as the last wave left it, not cleared

        def check(self, stream=None):
            abi.check(self.status(stream), "ib_batch_check")

        def close(self):
            pass

    return FakeBatch, made


@pytest.fixture
def fake(monkeypatch):
    from paper_2012_06646_gb300 import _abi, serve
    _abi.load()
    monkeypatch.setattr(torch.cuda, "Stream", FakeStream)
    monkeypatch.setattr(torch.cuda, "Event", FakeEvent)
    monkeypatch.setattr(torch.cuda, "synchronize", lambda *a, **k: None)

    def use(fail_at=None):
        FB, made = make_fake_batch(_abi, fail_at)
        monkeypatch.setattr(serve, "Batch", FB)
        return made
    return _abi, serve, use


def _req(serve, rid, N, n, seed, arrival=0.0):
    g = np.random.default_rng(seed)
    X = torch.from_numpy(g.random((n, 3)).astype(np.float32))
    G = torch.from_numpy(g.standard_normal((n, 3)).astype(np.float32))
    return serve.Request(rid=rid, N=N, X=X, G=G, arrival=arrival, U=torch.empty((n, 3)))


def test_rejects_cancels_and_flags_invalid_on_host(fake):
    abi, serve, use = fake
    use()
    srv = serve.Server(nstreams=2, max_jobs=4, max_points=1000, max_cells=4096, budget_bytes=1 << 30,
                       device=torch.device("cuda", 0))
    reqs = [_req(serve, i, 8 + 4 * (i % 3), 50 + 37 * i, i) for i in range(10)]
    reqs.append(_req(serve, 10, 8, 1001, 10))               # more points than a slot holds
    reqs.append(_req(serve, 11, 17, 10, 11))                # 4913 cells > 4096
    reqs.append(_req(serve, 12, 0, 10, 12))                 # invalid grid
    reqs[3].cancelled = True
    reqs[6].X[5, 2] = float("nan")
    st = srv.serve(reqs, realtime=False)
    assert [r.status for r in reqs[10:]] == [serve.REJECTED] * 3
    assert "points" in reqs[10].reason and "cells" in reqs[11].reason and "INVALID_ARG" in reqs[12].reason
    assert reqs[3].status == serve.CANCELLED
    assert reqs[6].status == serve.INVALID and torch.isnan(reqs[6].U[5]).all()
    done = [r for r in reqs if r.status == serve.DONE]
    assert len(done) == 8 and st.jobs == 8 and len(st.latencies_ms) == 8
    assert all(torch.equal(r.U, r.G) for r in done)
    assert st.outcomes == {serve.DONE: 8, serve.REJECTED: 3, serve.CANCELLED: 1, serve.INVALID: 1}
    # every wave respected the job cap, and the cancelled request never ran
    assert all(w <= 4 for b in srv.batches for w in b.waves)
    assert sum(w for b in srv.batches for w in b.waves) == 9


def test_cancelling_a_request_in_flight_reports_it_cancelled(fake):
    abi, serve, use = fake
    use()
    srv = serve.Server(nstreams=1, max_jobs=8, max_points=1 << 16, max_cells=1 << 16, budget_bytes=1 << 30,
                       device=torch.device("cuda", 0))
    reqs = [_req(serve, i, 8, 100, i) for i in range(3)]
    orig = srv._launch

    def launch_then_cancel(slot, wave, fp):
        w = orig(slot, wave, fp)
        srv.cancel(wave[0])                                  # cancelled after admission
        return w
    srv._launch = launch_then_cancel
    srv.serve(reqs, realtime=False)
    assert [r.status for r in reqs] == [serve.CANCELLED, serve.DONE, serve.DONE]


def test_server_runs_on_the_slots_it_could_allocate_on_host(fake):
    abi, serve, use = fake
    use(fail_at=2)
    srv = serve.Server(nstreams=4, max_jobs=4, max_points=1000, max_cells=4096, budget_bytes=1 << 30,
                       device=torch.device("cuda", 0))
    assert srv.nstreams == 2 and len(srv.batches) == 2 and len(srv.streams) == 2
    st = srv.serve([_req(serve, i, 8, 40, i) for i in range(6)], realtime=False)
    assert st.jobs == 6
    use(fail_at=0)
    with pytest.raises(abi.IBError) as e:
        serve.Server(nstreams=2, budget_bytes=1 << 30, device=torch.device("cuda", 0))
    assert e.value.status == abi.IB_ERR_OOM
