"""Host logic of bench.py's multi-GPU form, on CPU with the gloo backend.

Two ranks: each replica gets its own seed, the timed total is the maximum
over ranks, the job rate counts every rank's points over that time, and the
reference leg under torchrun prints exactly one line (rank 0).
"""
import json
import os
import socket
import subprocess
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        local_ms = [12.5, 40.0][rank]
        tot = bench.max_over_ranks(local_ms)
        out.put((rank, bench.rank_seed(7, rank), tot, bench.job_rate(1000, world, 10, tot)))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_and_rate_with_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, s0, t0, v0), (r1, s1, t1, v1) = res
    assert s0 != s1                              # independent replicas
    assert t0 == t1 == 40.0                      # slowest rank's time on every rank
    assert v0 == v1 == pytest.approx(1000 * 2 * 10 / 0.040)


def _shard_main(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    import ib_inputs
    from paper_2012_06646_gb300 import serve
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        specs = ib_inputs.job_mix(1, 384)
        owner = serve.place_jobs([sp.npts + sp.N ** 3 for sp in specs], world)
        mine = [i for i, o in enumerate(owner) if o == rank]
        shares = [None] * world
        dist.all_gather_object(shares, mine)
        wall = bench.max_over_ranks([0.25, 0.5][rank])
        out.put((rank, shares, wall, len(specs) / wall))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_served_jobs_shard_over_two_gloo_ranks():
    # Every rank computes the same placement on its own; the shares cover every job exactly once;
    # the capacity counts all jobs over the slowest rank's wall time.
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_shard_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, sh0, w0, c0), (r1, sh1, w1, c1) = res
    assert sh0 == sh1                                  # the same placement on both ranks
    assert sorted(sh0[0] + sh0[1]) == list(range(384)) and not set(sh0[0]) & set(sh0[1])
    assert w0 == w1 == 0.5 and c0 == c1 == pytest.approx(384 / 0.5)


def test_job_placement_balances_work():
    sys.path.insert(0, ROOT)
    import ib_inputs
    from paper_2012_06646_gb300 import serve
    specs = ib_inputs.job_mix(1, 384)
    cost = [sp.npts + sp.N ** 3 for sp in specs]
    assert serve.place_jobs(cost, 1) == [0] * len(cost)
    for world in (2, 3, 8):
        owner = serve.place_jobs(cost, world)
        assert owner == serve.place_jobs(cost, world)          # deterministic
        load = [sum(c for c, o in zip(cost, owner) if o == r) for r in range(world)]
        assert max(load) - min(load) <= max(cost)               # greedy longest-first bound
    assert serve.place_jobs([5, 1, 1, 1, 1, 1], 2) == [0, 1, 1, 1, 1, 1]
    with pytest.raises(ValueError):
        serve.place_jobs(cost, 0)


def test_single_rank_helpers():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.5) == 3.5
    assert bench.job_rate(10, 1, 4, 2.0) == pytest.approx(20000.0)
    assert bench.rank_seed(0, 0) == 0


def test_reference_leg_under_torchrun_prints_one_line():
    port = _free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node=2",
           "--master-addr=127.0.0.1", f"--master-port={port}", os.path.join(ROOT, "bench.py"),
           "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "1", "--grid", "16",
           "--points", "2000"]
    env = dict(os.environ, OMP_NUM_THREADS="1")
    res = subprocess.run(cmd, capture_output=True, text=True, timeout=300, cwd=ROOT, env=env)
    assert res.returncode == 0, res.stderr[-2000:]
    lines = [ln for ln in res.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    rec = json.loads(lines[0])
    assert rec["impl"] == "reference" and rec["n_gpus"] == 2 and rec["value"] > 0
    assert rec["cpu_baseline"]["kind"] == "oracle"
