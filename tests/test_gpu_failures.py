"""Host-side failure handling on the GPU path: arena allocation failures through
the allocator hook (IB_ERR_OOM, misaligned arenas, a server that loses a slot),
and the served loop's per-request outcomes for jobs that never fit a slot,
cancelled requests and non-finite positions.  No case faults, traps or stalls
the GPU: every failure is made on the host."""
import numpy as np
import pytest
import torch

import ib_inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mods():
    from paper_2012_06646_gb300 import build
    build()
    from paper_2012_06646_gb300 import _abi, plan, serve
    yield _abi, plan, serve
    plan.set_allocator()


class Counting:
    """PyTorch caching allocator behind counters; fails once `budget` arenas were handed out."""

    def __init__(self, budget=None, offset=0):
        self.budget, self.offset = budget, offset
        self.live, self.allocs, self.frees = {}, 0, []

    def alloc(self, n):
        if self.budget is not None and self.allocs >= self.budget:
            return 0
        p = torch.cuda.caching_allocator_alloc(n + self.offset)
        self.allocs += 1
        self.live[p + self.offset] = p
        return p + self.offset

    def free(self, q):
        self.frees.append(q)
        torch.cuda.caching_allocator_delete(self.live.pop(q))


def _points(seed, n, N):
    g = np.random.default_rng(seed)
    X = torch.from_numpy(g.random((n, 3)).astype(np.float32)).cuda()
    G = torch.from_numpy(g.standard_normal((n, 3)).astype(np.float32)).cuda()
    return X, G


def test_failing_allocator_gives_oom_and_holds_nothing(mods):
    _abi, plan, serve = mods
    c = Counting(budget=0)
    plan.set_allocator(c.alloc, c.free)
    try:
        with pytest.raises(_abi.IBError) as e:
            plan.Plan(3, (16, 16, 16), (1.0, 1.0, 1.0), max_points=100)
        assert e.value.status == _abi.IB_ERR_OOM
        with pytest.raises(_abi.IBError) as e:
            plan.Batch(dim=3, max_jobs=4, max_points=1 << 12, max_cells=1 << 15, host_io=True)
        assert e.value.status == _abi.IB_ERR_OOM
        # an exception inside alloc counts as out of memory too
        plan.set_allocator(lambda n: 1 // 0, c.free)
        with pytest.raises(_abi.IBError) as e:
            plan.Plan(3, (16, 16, 16), (1.0, 1.0, 1.0), max_points=100)
        assert e.value.status == _abi.IB_ERR_OOM
    finally:
        plan.set_allocator()
    assert c.frees == []
    # the default allocator works again
    p = plan.Plan(3, (16, 16, 16), (1.0, 1.0, 1.0), max_points=100)
    p.close()


def test_misaligned_arena_is_returned_and_rejected(mods):
    _abi, plan, serve = mods
    c = Counting(offset=16)
    plan.set_allocator(c.alloc, c.free)
    try:
        with pytest.raises(_abi.IBError) as e:
            plan.Plan(3, (16, 16, 16), (1.0, 1.0, 1.0), max_points=100)
        assert e.value.status == _abi.IB_ERR_INVALID_ARG
    finally:
        plan.set_allocator()
    assert c.allocs == 1 and len(c.frees) == 1 and c.live == {}


def test_torch_allocator_arena_gives_identical_results(mods):
    _abi, plan, serve = mods
    N, n = 48, 20000
    X, G = _points(3, n, N)
    ref = plan.Plan(3, (N, N, N), (1.0, 1.0, 1.0), max_points=n)
    f0 = ref.spread(X, G)
    U0 = ref.interpolate(X, f0, reuse_bins=True)
    c = Counting()
    plan.set_allocator(c.alloc, c.free)
    try:
        p = plan.Plan(3, (N, N, N), (1.0, 1.0, 1.0), max_points=n)
    finally:
        plan.set_allocator()               # p keeps the pair it was created with
    f1 = p.spread(X, G)
    U1 = p.interpolate(X, f1, reuse_bins=True)
    p.check()
    assert torch.equal(f0, f1) and torch.equal(U0, U1)
    assert c.allocs == 1 and c.frees == []
    p.close()
    assert len(c.frees) == 1 and c.live == {}
    ref.close()
    plan.use_torch_allocator()
    try:
        p = plan.Plan(3, (N, N, N), (1.0, 1.0, 1.0), max_points=n)
        assert torch.equal(p.spread(X, G), f0)
        p.close()
    finally:
        plan.set_allocator()


def test_server_runs_on_the_slots_it_could_allocate(mods):
    _abi, plan, serve = mods
    c = Counting(budget=2)
    plan.set_allocator(c.alloc, c.free)
    try:
        srv = serve.Server(nstreams=3, max_jobs=8, max_points=1 << 14, max_cells=1 << 16)
    finally:
        plan.set_allocator()
    assert srv.nstreams == 2 and len(srv.streams) == 2
    specs = ib_inputs.job_mix(21, 10, grids=(8, 16, 24), n_lo=50, n_hi=2000)
    reqs = serve.make_requests(specs)
    st = srv.serve(reqs, realtime=False)
    assert st.jobs == 10 and all(r.status == serve.DONE for r in reqs)
    srv.close()
    assert len(c.frees) == 2 and c.live == {}


@pytest.mark.timeout(300)
def test_server_rejects_cancels_and_flags_invalid_positions(mods):
    _abi, plan, serve = mods
    specs = ib_inputs.job_mix(23, 12, grids=(8, 16, 24), n_lo=50, n_hi=1500)
    reqs = serve.make_requests(specs)
    rid = len(reqs)
    # a job with more points than a slot holds: rejected on arrival, not queued forever
    big = torch.rand((5000, 3), dtype=torch.float32).pin_memory()
    reqs.append(serve.Request(rid=rid, N=16, X=big, G=torch.ones_like(big).pin_memory()))
    # a grid with more cells than a slot holds
    reqs.append(serve.Request(rid=rid + 1, N=64, X=big[:10].clone().pin_memory(),
                              G=torch.ones((10, 3)).pin_memory()))
    # an invalid grid description
    reqs.append(serve.Request(rid=rid + 2, N=0, X=big[:10].clone().pin_memory(),
                              G=torch.ones((10, 3)).pin_memory()))
    reqs[2].cancelled = True                      # cancelled before it is admitted
    bad = reqs[5]
    bad.X[7, 1] = float("nan")                    # one non-finite position
    srv = serve.Server(nstreams=2, max_jobs=8, max_points=1 << 12, max_cells=1 << 15)
    st = srv.serve(reqs, realtime=False)
    srv.close()
    assert [r.status for r in reqs[-3:]] == [serve.REJECTED] * 3
    assert "points" in reqs[-3].reason and "cells" in reqs[-2].reason and reqs[-1].reason
    assert reqs[2].status == serve.CANCELLED
    assert bad.status == serve.INVALID
    assert torch.isnan(bad.U[7]).all()
    done = [r for r in reqs if r.status == serve.DONE]
    assert len(done) == 10 and st.jobs == 10
    assert st.outcomes == {serve.DONE: 10, serve.REJECTED: 3, serve.CANCELLED: 1, serve.INVALID: 1}
    # the jobs that ran alongside the invalid one are unaffected
    ref = serve.make_requests([specs[i] for i, r in enumerate(reqs[:12]) if r.status == serve.DONE])
    serve.single_job_loop(ref, realtime=False)
    for r, q in zip(done, ref):
        assert torch.equal(r.U, q.U)
