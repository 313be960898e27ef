"""Benchmark: spread + interpolate throughput on the 128^3 MAC grid with 10^6 points.

One step (the unstructured-point protocol of the paper's Section 4.1, reduced
to one spread and one interpolation): bin X, spread the step's forces G from X
onto the grid, interpolate the shear velocity u back to X, and move X by
dt U (dt chosen so the largest displacement is h/2).  `value` counts
Lagrangian points processed per second by that spread + interpolate pair.

Timing: W warm-up steps, then K timed steps, each bracketed by CUDA events on
the launching stream; L2 is flushed (256 MB write) between timed steps,
outside the events.  The timed step is one CUDA graph replay of the same
calls (captured once per force buffer, so the forces change every step;
--no-graph times the separate calls instead).  A first pass of W + K steps as
separate calls gives the per-call durations used for the breakdown and the
roofline.  `e2e` repeats the step through the same C ABI with host
buffers: X and G copied in from pinned memory and U, f and the new X copied
back every step, inside the timed region; the K steps stream back to back,
uploads and downloads on their own streams ordered by events, so a step's
downloads overlap the next step's kernels (`value_step_by_step` times each
step alone, `value_copies_serialised` with every copy in line).

--impl reference runs the FP64 CPU oracle on a bounded sample of the same
workload (rank 0 only).  Under torchrun each rank runs its own independent
replica of the workload (weak scaling, no data-path collective); rank 0
prints the max-over-ranks time.
"""

from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "spread+interp Lagrangian pts/s @128^3 vs HBM roofline; batched p50/p99 latency"
N_GRID = 128
N_POINTS = 1_000_000
GAMMA = 1.0


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--points", type=int, default=N_POINTS)
    ap.add_argument("--grid", type=int, default=N_GRID)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-sample", type=int, default=100_000)
    ap.add_argument("--clock-window", type=float, default=1.0,
                    help="seconds of clock sampling from the start of the timed steps")
    ap.add_argument("--serve-jobs", type=int, default=4096, help="jobs of the served-batch measurement (0: skip)")
    ap.add_argument("--serve-loads", default="0.5,0.9,1.5",
                    help="offered loads as multiples of the one-job loop's capacity, comma separated")
    ap.add_argument("--no-graph", action="store_true",
                    help="time the step as separate calls instead of one CUDA graph replay")
    ap.add_argument("--membrane-reps", type=int, default=10,
                    help="timed repetitions of the clustered red-cell membrane workload (0: skip)")
    ap.add_argument("--paper-reps", type=int, default=3,
                    help="timed repetitions of the paper's spreading algorithms 4-6 on the workload (0: skip)")
    ap.add_argument("--grad-reps", type=int, default=10,
                    help="timed repetitions of the differentiable spread (forward and backward; 0: skip)")
    ap.add_argument("--kernel-reps", type=int, default=10,
                    help="timed repetitions of spread + interpolate with each other kernel (0: skip)")
    ap.add_argument("--ib-step-reps", type=int, default=10,
                    help="timed repetitions of the full IB timestep (a)-(g) with the Stokes solve (0: skip)")
    return ap.parse_args()


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def rank_seed(seed: int, rank: int) -> int:
    """Seed of a rank's independent replica of the workload."""
    return seed + 7919 * rank


def max_over_ranks(x: float, device=None) -> float:
    """Largest value of x over all ranks (x itself on one rank)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(units_per_rank: int, world: int, steps: int, total_ms: float) -> float:
    """Whole-job throughput: units processed by all ranks over the slowest rank's time."""
    return units_per_rank * world * steps / (total_ms / 1e3)


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            p = json.load(fh)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# Sources of the kernels whose DRAM counters profiles/traffic.txt records (the
# spreading and interpolation kernels and the device header they include).
TRAFFIC_SOURCES = ("ib_ops.cu", "ib_common.cuh")


def csrc_hash():
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_2012_06646_gb300", "csrc")
    for name in TRAFFIC_SOURCES:
        with open(os.path.join(d, name), "rb") as fh:
            h.update(name.encode() + fh.read())
    return h.hexdigest()[:16]


def step_distribution(ms: list):
    """p50 / p99 / min / max / mean of this rank's timed step durations (ms)."""
    if not ms:
        return None
    a = np.asarray(ms, dtype=np.float64)
    return {"p50": float(np.percentile(a, 50)), "p99": float(np.percentile(a, 99)), "min": float(a.min()),
            "max": float(a.max()), "mean": float(a.mean()), "n": int(a.size)}


def output_hash(*tensors) -> str:
    """First 16 hex digits of a SHA-256 over the bytes of the given tensors (the step's outputs):
    equal across runs of the same configuration, since every sum has a fixed order."""
    h = hashlib.sha256()
    for t in tensors:
        h.update(t.detach().cpu().numpy().tobytes())
    return h.hexdigest()[:16]


def ncu_traffic(kernel: str):
    """DRAM bytes per launch of `kernel` from the committed ncu summary, if it was
    captured on the current kernel sources (else None)."""
    path = os.path.join(ROOT, "profiles", "traffic.txt")
    if not os.path.exists(path):
        return None
    src, val = None, None
    with open(path) as fh:
        for line in fh:
            parts = line.split()
            if len(parts) >= 2 and parts[0] == "csrc_sha256_16:":
                src = parts[1]
            if len(parts) >= 2 and parts[0] == f"{kernel}_dram_bytes_per_launch:":
                val = float(parts[1])
    return val if (src == csrc_hash() and val is not None) else None


class ClockSampler:
    """nvidia-smi clock / throttle sampling.  Each sample is stamped on arrival,
    so the summary covers exactly the window it is asked for."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id: str):
        self.gpu = gpu_id
        self.proc = None
        self.rows = []
        self.thread = None

    def start(self, wait_s: float = 5.0):
        import threading
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return

        def reader():
            for line in self.proc.stdout:
                self.rows.append((time.time(), line))

        self.thread = threading.Thread(target=reader, daemon=True)
        self.thread.start()
        t0 = time.time()
        while not self.rows and time.time() - t0 < wait_s and self.proc.poll() is None:
            time.sleep(0.01)

    def stop(self, t_begin: float, t_end: float):
        if self.proc is None:
            return None
        time.sleep(0.15)                 # the sample taken at t_end arrives shortly after
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        if self.thread is not None:
            self.thread.join(timeout=2)
        rows = []
        for t, line in self.rows:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9 and t_begin <= t <= t_end + 0.1:
                rows.append(parts)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def workload(seed, npts, N):
    import ib_inputs
    X = ib_inputs.uniform_points(seed, npts, (1.0, 1.0, 1.0), 3)
    u = ib_inputs.shear_field_mac(N, 1.0, GAMMA)
    return X, u


def forces(seed, step, npts):
    import ib_inputs
    return ib_inputs.normal_array(seed * 1000 + step, (npts, 3), purpose="G")


def cpu_oracle_rate(sample: int, N: int, seed: int, kernel: int = 0, bounded=()):
    """The FP64 oracle (single thread) on `sample` points of the workload:
    one spread + one interpolation; returns (pts/s, seconds)."""
    import oracle
    X, u = workload(seed, sample, N)
    G = forces(seed, 0, sample)
    g = oracle.Grid(dim=3, n=(N, N, N), L=(1.0, 1.0, 1.0), mac=True, kernel=kernel, bounded=bounded)
    t0 = time.perf_counter()
    oracle.spread(g, X, G)
    oracle.interp(g, X, u)
    dt = time.perf_counter() - t0
    return sample / dt, dt


# The oracle over all host cores: spawned worker processes (no CUDA in them),
# each with its share of the points; interpolation is independent per point,
# and each worker spreads its share into its own FP64 grid in shared memory,
# summed in worker order afterwards.
_PAR = {}


def _par_init(seed, N, npts, shm_name, procs, barrier):
    from multiprocessing import shared_memory
    import oracle
    oracle.lib()
    X, u = workload(seed, npts, N)
    _PAR.update(X=X, u=u, G=forces(seed, 0, npts), N=N, procs=procs,
                shm=shared_memory.SharedMemory(name=shm_name))
    barrier.wait(timeout=60)


def _par_work(k):
    import oracle
    P = _PAR
    N = P["N"]
    part = np.array_split(np.arange(len(P["X"])), P["procs"])[k]
    g = oracle.Grid(dim=3, n=(N, N, N), L=(1.0, 1.0, 1.0), mac=True)
    f, _ = oracle.spread(g, P["X"][part], P["G"][part])
    np.ndarray((P["procs"], 3 * N ** 3), dtype=np.float64, buffer=P["shm"].buf)[k] = f.ravel()
    U, _ = oracle.interp(g, P["X"][part], P["u"])
    return U


def cpu_oracle_parallel(N: int, seed: int, npts: int):
    """The FP64 oracle as it stands, one spread + one interpolation of all npts
    points, split over every host core; returns (pts/s, seconds, cores)."""
    import multiprocessing as mp
    from multiprocessing import shared_memory
    procs = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)
    ctx = mp.get_context("spawn")
    shm = shared_memory.SharedMemory(create=True, size=procs * 3 * N ** 3 * 8)
    try:
        barrier = ctx.Barrier(procs + 1)
        # A worker that cannot start breaks the barrier: the wait times out, and
        # leaving the block terminates the pool.
        with ctx.Pool(procs, initializer=_par_init, initargs=(seed, N, npts, shm.name, procs, barrier)) as pool:
            barrier.wait(timeout=60)                         # every worker holds its inputs
            t0 = time.perf_counter()
            parts = pool.map_async(_par_work, range(procs), chunksize=1).get(timeout=600)
            grids = np.ndarray((procs, 3 * N ** 3), dtype=np.float64, buffer=shm.buf)
            f = grids[0].copy()
            for k in range(1, procs):
                f += grids[k]
            U = np.concatenate(parts)
            dt = time.perf_counter() - t0
            del grids
        assert U.shape == (npts, 3) and np.isfinite(f).all()
    finally:
        shm.close()
        shm.unlink()
    return npts / dt, dt, procs


def serving_bench(device, njobs: int, loads, seed: int = 1, world: int = 1, rank: int = 0):
    """Served batch: independent spread + interpolate jobs, N in {32, 64, 96, 128}, n log-uniform in
    [1e3, 1e5], half uniform / half on RBC shells.  The one-job-per-launch loop is first run back to
    back to measure its capacity, and the continuous-batching server likewise; then Poisson arrivals
    at each offered load (a multiple of the loop's capacity) are served by the server and by the
    loop.  Latency = completion - arrival.  Under torchrun the jobs are sharded over the ranks
    (serve.place_jobs, no data-path collective): each rank serves its own share, the capacities
    count every rank's jobs over the slowest rank's wall time, and the latencies are rank 0's."""
    import ib_inputs
    import torch
    from paper_2012_06646_gb300 import serve
    all_specs = ib_inputs.job_mix(seed, njobs)
    owner = serve.place_jobs([sp.npts + sp.N ** 3 for sp in all_specs], world)
    specs = [sp for sp, o in zip(all_specs, owner) if o == rank]
    share = len(specs)
    warm = serve.make_requests(specs[: min(16, share)])
    serve.single_job_loop(warm, realtime=False, device=device)
    srv = serve.Server(nstreams=3, max_jobs=64, max_points=1 << 22, max_cells=1 << 25, device=device)
    srv.serve(serve.make_requests(specs[: min(16, share)]), realtime=False)
    reqs = serve.make_requests(specs)
    cap_loop = serve.single_job_loop(reqs, realtime=False, device=device)
    loop_U = [r.U.clone() for r in reqs]
    cap_srv = srv.serve(reqs, realtime=False)
    same = all(torch.equal(a, r.U) for a, r in zip(loop_U, reqs))
    cap = cap_loop.jobs / cap_loop.wall_s           # this rank's loop capacity (sets its offered loads)
    wall_loop = max_over_ranks(cap_loop.wall_s, device)
    wall_srv = max_over_ranks(cap_srv.wall_s, device)
    same = max_over_ranks(0.0 if same else 1.0, device) == 0.0
    out = {"jobs": njobs, "points": int(sum(sp.npts for sp in all_specs)),
           "capacity_jobs_per_s": {"single_job_loop": njobs / wall_loop, "batched": njobs / wall_srv},
           "results_identical_alone_and_in_mix": bool(same), "loads": []}
    if world > 1:
        out["sharding"] = {"ranks": world, "placement": "longest job first onto the least-loaded rank "
                                                       "(cost = points + grid cells); no data-path collective",
                           "jobs_rank0": share, "latencies": "rank 0's share, offered at the load times "
                                                               "rank 0's own loop capacity"}
    for load in loads:
        arrivals = ib_inputs.poisson_arrivals(seed, share, load * cap)
        for r, t in zip(reqs, arrivals):
            r.arrival, r.t_done = float(t), -1.0
        st_b = srv.serve(reqs)
        for r in reqs:
            r.t_done = -1.0
        st_l = serve.single_job_loop(reqs, device=device)
        out["loads"].append({"offered_load_x_loop_capacity": load, "offered_jobs_per_s": load * cap,
                             "batched": st_b.summary(), "single_job_loop": st_l.summary()})
    srv.close()
    return out


def run_reference(args):
    world, rank, _ = dist_env()
    if rank != 0:
        return
    import oracle
    oracle.build()
    sample = max(1000, min(args.points, 30_000))
    N = args.grid
    X, u = workload(args.seed, sample, N)
    g = oracle.Grid(dim=3, n=(N, N, N), L=(1.0, 1.0, 1.0), mac=True)
    h = 1.0 / N
    dt = h / (GAMMA * 1.0)
    times = []
    for step in range(args.warmup + args.steps):
        G = forces(args.seed, step, sample)
        t0 = time.perf_counter()
        oracle.spread(g, X, G)
        U, _ = oracle.interp(g, X, u)
        X = (X.astype(np.float64) + dt * U)
        X = (X - np.floor(X)).astype(np.float32)
        t = time.perf_counter() - t0
        if step >= args.warmup:
            times.append(t)
    tot = sum(times)
    value = sample * len(times) / tot
    cores = 1
    line = {"metric": METRIC, "value": value, "unit": "pts/s", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * tot / len(times), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {"workload": f"{N}^3 MAC grid, uniform points, one spread + one interpolation + advection "
                                   f"per step (bounded sample of {sample} of the {args.points} points)",
                       "grid": N, "n_points": args.points, "sample_points": sample},
            "cpu_baseline": {"value": value, "unit": "pts/s", "cores": cores, "kind": "oracle",
                             "sample": f"{sample} points per step, FP64 direct sums, single thread"},
            "e2e": {"value": value, "unit": "pts/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def paper_algorithms_bench(plan, X, G, f, stream, reps, beta=8):
    """The paper's spreading algorithms 4, 5 and 6 (beta shifts per pass) next to
    this library's binning + spreading, on the same points and forces: mean
    milliseconds per call over `reps` timed calls after one warm-up call, L2
    flushed before each.  Every variant includes its own key computation and sort."""
    import torch
    device = X.device
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=device)
    buf = torch.empty((beta,) + tuple(reversed(plan.n)), dtype=torch.float32, device=device)
    variants = {
        "ours_bin_and_spread": lambda: (plan.bin(X, stream=stream), plan.spread(X, G, f=f, reuse_bins=True,
                                                                                stream=stream)),
        "alg4": lambda: plan.spread_paper(X, G, algorithm=4, f=f, stream=stream),
        f"alg5_beta{beta}": lambda: plan.spread_paper(X, G, algorithm=5, beta=beta, f=f, buffer=buf, stream=stream),
        f"alg6_beta{beta}": lambda: plan.spread_paper(X, G, algorithm=6, beta=beta, f=f, stream=stream),
    }
    out = {}
    with torch.cuda.stream(stream):
        for name, call in variants.items():
            call()
            times = []
            for r in range(reps):
                flush.fill_(r & 0xFF)
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                call()
                b.record(stream)
                b.synchronize()
                times.append(a.elapsed_time(b))
            out[name + "_ms"] = statistics.mean(times)
    plan.check(stream)
    base = out["ours_bin_and_spread_ms"]
    out["speedup_over"] = {k[:-3]: v / base for k, v in out.items() if k != "ours_bin_and_spread_ms"}
    return out


def touched_nodes_mac(X: np.ndarray, N: int) -> int:
    """Distinct grid nodes (summed over the three MAC components) inside the 4^3
    support of at least one point: the nodes a spread writes or an interpolation
    reads when only the touched part of the grid counts."""
    total = 0
    u = X.astype(np.float64) * N
    t = np.arange(4) - 1
    for a in range(3):
        base = np.floor(u - np.where(np.arange(3) == a, 0.0, 0.5)).astype(np.int64)   # cell of this staggering
        ix = (base[:, None, 0] + t[None, :]) % N
        iy = (base[:, None, 1] + t[None, :]) % N
        iz = (base[:, None, 2] + t[None, :]) % N
        idx = (ix[:, :, None, None] + N * (iy[:, None, :, None] + N * iz[:, None, None, :])).ravel()
        total += int(np.unique(idx).size)
    return total


FLOOR32 = 64 * 1.1754943508222875e-38      # 64 FLT_MIN: contributions below the FP32 normal range


def error_vs_oracle(got, ref, absref, floor: float = FLOOR32) -> dict:
    """Worst relative error of a GPU result against the FP64 oracle, in the tests'
    measure: |got - ref| / (sum |terms| + floor) per node or point (the sum of
    |terms| is the oracle's sum of |contribution|), with the tolerance it must meet."""
    got = np.asarray(got, dtype=np.float64)
    err = np.abs(got - ref)
    rel = err / (absref + floor)
    return {"max_rel_err": float(rel.max()) if rel.size else 0.0,
            "mean_rel_err": float(rel.mean()) if rel.size else 0.0,
            "sum_abs_err": float(err.sum()), "count": int(rel.size), "tolerance": 1e-5,
            "within_tolerance": bool(np.all(err <= 1e-5 * absref + floor))}


def membrane_bench(device, stream, reps: int, peak: float, seed: int = 0, N: int = 128, oracle_check: bool = True):
    """The clustered-membrane workload: 17 randomly oriented, non-overlapping red
    cells compressed to about 40 % volume fraction in the 128^3 MAC box, with
    2562 points per cell and with the paper's 8832, smooth membrane forces.
    Times binning + spreading (TwoSum node sums, and plain) and interpolation,
    CUDA events on the stream, L2 flushed before each timed call; then (outside
    the timing) states the error of each result against the FP64 oracle."""
    import torch
    import ib_inputs
    from paper_2012_06646_gb300.plan import Plan
    out = {}
    for label, per_cell in (("rbc2562", None), ("rbc8832", 8832)):
        mem = ib_inputs.pack_membranes(seed, points_per_cell=per_cell)
        Gh = ib_inputs.membrane_forces(seed, mem)
        uh = ib_inputs.normal_array(seed + 1, (3, N, N, N))
        X = torch.from_numpy(mem.X).to(device)
        G = torch.from_numpy(Gh).to(device)
        u = torch.from_numpy(uh).to(device)
        n = X.shape[0]
        plan = Plan(3, (N, N, N), (1.0, 1.0, 1.0), grid="mac", max_points=n, compensated=True, device=device)
        f = torch.empty(plan.grid_shape(), dtype=torch.float32, device=device)
        U = torch.empty((n, 3), dtype=torch.float32, device=device)
        flush = torch.empty(256 << 20, dtype=torch.uint8, device=device)
        calls = {
            "bin_and_spread_compensated": lambda: plan.spread(X, G, f=f, compensated=True, stream=stream),
            "bin_and_spread": lambda: plan.spread(X, G, f=f, stream=stream),
            "interp": lambda: plan.interpolate(X, u, U=U, reuse_bins=True, stream=stream),
        }
        ms = {}
        with torch.cuda.stream(stream):
            for name, call in calls.items():
                call()
                t = []
                for r in range(reps):
                    flush.fill_(r & 0xFF)
                    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    a.record(stream)
                    call()
                    b.record(stream)
                    b.synchronize()
                    t.append(a.elapsed_time(b))
                ms[name] = statistics.mean(t)
        plan.check(stream)
        pair = ms["bin_and_spread_compensated"] + ms["interp"]
        grid_bytes = 2 * (n * 24 + 3 * N ** 3 * 4)
        touched = touched_nodes_mac(mem.X, N)
        touched_bytes = 2 * (n * 24 + touched * 4)
        res = {"workload": f"{len(mem.centres)} red cells x {n // max(1, len(mem.centres))} points ({n} points, "
                           f"volume fraction {mem.volume_fraction:.3f}), {N}^3 MAC grid, FP32, TwoSum node sums "
                           "in spreading",
               "calls_ms": ms, "pts_per_s": n / (pair / 1e3),
               "roofline_full_grid": {"achieved_gbs": grid_bytes / (pair / 1e3) / 1e9, "peak": peak,
                                      "frac": grid_bytes / (pair / 1e3) / 1e9 / peak, "bytes": grid_bytes},
               "roofline_touched_nodes": {"achieved_gbs": touched_bytes / (pair / 1e3) / 1e9, "peak": peak,
                                          "frac": touched_bytes / (pair / 1e3) / 1e9 / peak, "bytes": touched_bytes,
                                          "touched_nodes": touched},
               "note": "spread + interpolate pair (compensated spread, binning included)"}
        if oracle_check:
            import oracle
            oracle.build()
            with torch.cuda.stream(stream):
                fc = plan.spread(X, G, compensated=True, stream=stream).cpu().numpy()
                fp = plan.spread(X, G, reuse_bins=True, stream=stream).cpu().numpy()
                Ug = plan.interpolate(X, u, reuse_bins=True, stream=stream).cpu().numpy()
            g = oracle.Grid(dim=3, n=(N, N, N), L=(1.0, 1.0, 1.0), mac=True)
            f_ref, fabs = oracle.spread(g, mem.X, Gh)
            U_ref, Uabs = oracle.interp(g, mem.X, uh)
            ec, ep = error_vs_oracle(fc, f_ref, fabs), error_vs_oracle(fp, f_ref, fabs)
            res["error_vs_fp64_oracle"] = {
                "spread_compensated": ec, "spread_plain": ep, "interp": error_vs_oracle(Ug, U_ref, Uabs),
                "compensated_over_plain_sum_abs_err": ec["sum_abs_err"] / ep["sum_abs_err"] if ep["sum_abs_err"] else None,
                "measure": "per node |f - f_ref| / (sum |terms| + 64 FLT_MIN), per point likewise; every node and point"}
        out[label] = res
    return out


def accuracy_uniform(plan, X, G, u, N: int, stream, seed: int = 0, sample: int = 20_000, box: int = 24) -> dict:
    """Error of the headline workload's spreading and interpolation against the FP64
    oracle, outside the timing.  Interpolation: a sample of points, each against
    the oracle's own sum.  Spreading: the nodes of an interior sub-box of box^3
    cells, against the oracle's spread of every point whose support reaches
    them (points with floor(X N) within 3 cells of the sub-box), which gives
    those nodes their complete sums."""
    import torch
    import oracle
    oracle.build()
    with torch.cuda.stream(stream):
        f = plan.spread(X, G, stream=stream).cpu().numpy()
        U = plan.interpolate(X, u, reuse_bins=True, stream=stream).cpu().numpy()
    Xh = X.cpu().numpy()
    Gh = G.cpu().numpy()
    uh = u.cpu().numpy()
    g = oracle.Grid(dim=3, n=(N, N, N), L=(1.0, 1.0, 1.0), mac=True)
    pick = np.linspace(0, len(Xh) - 1, min(sample, len(Xh))).astype(np.int64)
    U_ref, Uabs = oracle.interp(g, Xh[pick], uh)
    c0 = N // 3
    cells = np.floor(Xh.astype(np.float64) * N).astype(np.int64)
    sel = np.all((cells >= c0 - 3) & (cells <= c0 + box + 2), axis=1)
    f_ref, fabs = oracle.spread(g, Xh[sel], Gh[sel])
    w = np.s_[:, c0:c0 + box, c0:c0 + box, c0:c0 + box]
    return {"spread": dict(error_vs_oracle(f[w], f_ref[w], fabs[w]),
                           nodes=f"{box}^3 interior nodes x 3 components from {int(sel.sum())} points"),
            "interp": dict(error_vs_oracle(U[pick], U_ref, Uabs), points=f"{len(pick)} evenly spaced points"),
            "measure": "per node |f - f_ref| / (sum |terms| + 64 FLT_MIN), per point likewise"}


def kernels_bench(device, stream, X, G, u, reps: int, N: int, peak: float, oracle_sample: int = 0):
    """Bin + spread + interpolate on the bench workload with every kernel of
    the library (support widths 4, 4, 3, 6): CUDA events on the stream, L2
    flushed before each timed repetition.  Each line carries the pair's HBM
    roofline fraction (the algorithmic bytes of the headline pair) and, with
    oracle_sample > 0, the FP64 oracle's single-thread rate on that many points."""
    import torch
    from paper_2012_06646_gb300.plan import Plan
    npts = X.shape[0]
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=device)
    out = {}
    cases = (("peskin4", 4, False), ("cosine4", 4, False), ("roma3", 3, False), ("bspline6", 6, False),
             ("peskin4", 4, True))
    for name, width, walls in cases:
        plan = Plan(3, (N, N, N), (1.0, 1.0, 1.0), grid="mac", kernel=name, max_points=npts, device=device,
                    bounded=(False, False, walls))
        f = torch.empty(plan.grid_shape(), dtype=torch.float32, device=device)
        U = torch.empty((npts, 3), dtype=torch.float32, device=device)
        ms = {"spread": [], "interp": []}
        with torch.cuda.stream(stream):
            for r in range(reps + 2):
                flush.fill_(r & 0xFF)
                e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
                e[0].record(stream)
                plan.spread(X, G, f=f, stream=stream)
                e[1].record(stream)
                plan.interpolate(X, u, U=U, reuse_bins=True, stream=stream)
                e[2].record(stream)
                e[2].synchronize()
                if r >= 2:
                    ms["spread"].append(e[0].elapsed_time(e[1]))
                    ms["interp"].append(e[1].elapsed_time(e[2]))
        plan.check(stream)
        plan.close()
        sp, it = statistics.mean(ms["spread"]), statistics.mean(ms["interp"])
        pair_bytes = 2 * (npts * 24 + 3 * N ** 3 * 4)
        line = {"support": width, "bin_and_spread_ms": sp, "interp_ms": it, "pts_per_s": npts / ((sp + it) / 1e3),
                "roofline_frac": pair_bytes / ((sp + it) / 1e3) / 1e9 / peak}
        if oracle_sample > 0:
            kid = {"peskin4": 0, "cosine4": 1, "roma3": 2, "bspline6": 3}[name]
            rate, secs = cpu_oracle_rate(oracle_sample, N, 0, kid, (False, False, walls))
            line["oracle_pts_per_s"] = rate
        out[name + ("_walls_z" if walls else "")] = line
    return {"workload": f"{N}^3 MAC grid, {npts} uniform points, FP32, spread (binning included) + interpolate; "
                        "'_walls_z': non-periodic in z (walls at z = 0 and z = L)",
            "roofline": f"pair bytes 2 (24 n + 12 N^3) / (spread + interp time) over {peak} GB/s (measured HBM)",
            "oracle": f"FP64 oracle, one thread, {oracle_sample} points of the workload, spread + interpolate",
            "kernels": out}


def autograd_bench(device, stream, reps: int, N: int, npts: int = 200_000, seed: int = 5):
    """The differentiable workload: 128^3 MAC grid, 2 x 10^5 uniform points,
    f = spread(X, G) through the autograd Function, loss = sum(w f) with
    w ~ N(0, 1), then loss.backward(): binning, the adjoint interpolation
    (dloss/dG) and the position gradient (dloss/dX).  CUDA events on the
    stream around forward + backward, L2 flushed before each repetition."""
    import torch
    import ib_inputs
    from paper_2012_06646_gb300 import autograd as ag
    from paper_2012_06646_gb300.plan import Plan
    X = torch.from_numpy(ib_inputs.uniform_points(seed, npts, (1.0, 1.0, 1.0), 3)).to(device).requires_grad_(True)
    G = torch.from_numpy(ib_inputs.normal_array(seed + 1, (npts, 3))).to(device).requires_grad_(True)
    w = torch.from_numpy(ib_inputs.normal_array(seed + 2, (3, N, N, N))).to(device)
    plan = Plan(3, (N, N, N), (1.0, 1.0, 1.0), grid="mac", max_points=npts, device=device)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=device)
    ms = []
    with torch.cuda.stream(stream):
        for r in range(reps + 2):
            flush.fill_(r & 0xFF)
            X.grad = None
            G.grad = None
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            f = ag.spread(X, G, plan)
            loss = (w * f).sum()
            loss.backward()
            b.record(stream)
            b.synchronize()
            if r >= 2:
                ms.append(a.elapsed_time(b))
    plan.check(stream)
    ok = bool(torch.isfinite(X.grad).all().item() and torch.isfinite(G.grad).all().item())
    # The same forward and backward captured once as a CUDA graph (the
    # library's calls are stream-ordered launches), replayed per repetition.
    gms = []
    with torch.cuda.stream(stream):
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph, stream=stream):
            fg = ag.spread(X, G, plan)
            gX, gG = torch.autograd.grad((w * fg).sum(), (X, G))
        for r in range(reps + 2):
            flush.fill_(r & 0xFF)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            graph.replay()
            b.record(stream)
            b.synchronize()
            if r >= 2:
                gms.append(a.elapsed_time(b))
    plan.check(stream)
    same = bool(torch.equal(gX, X.grad) and torch.equal(gG, G.grad))
    plan.close()
    t, tg = statistics.mean(ms), statistics.mean(gms)
    return {"workload": f"{N}^3 MAC grid, {npts} uniform points, FP32; f = spread(X, G), loss = sum(w f), "
                        "backward: dloss/dG by adjoint interpolation, dloss/dX by the position gradient",
            "step_ms": t, "pts_per_s": npts / (t / 1e3), "gradients_finite": ok,
            "step_ms_cuda_graph": tg, "pts_per_s_cuda_graph": npts / (tg / 1e3),
            "graph_gradients_equal_eager": same}


def ib_step_bench(device, stream, X0, ud, G, reps: int, peak: float, N: int, dt: float,
                  rho: float = 1.0, mu: float = 1.0e-2, oracle_solve: bool = True):
    """The full IB timestep (Section 2, steps (a)-(g)) on the bench workload:
    bin + interpolate, advect, bin + spread the given forces (step (c), the
    elastic model, is outside the library: the forces are a fixed buffer),
    the periodic Stokes solve, interpolate, advect.  CUDA events on the
    stream, L2 flushed before each timed step; the Stokes solve is also timed
    alone, against its algorithmic bytes (read f and u_old, write u)."""
    import torch
    from paper_2012_06646_gb300.step import IBStep
    npts = X0.shape[0]
    stepper = IBStep(3, (N, N, N), (1.0, 1.0, 1.0), rho, mu, dt, max_points=npts, device=device)
    X = X0.clone()
    Xo = torch.empty_like(X)
    u_a = ud.clone()
    u_b = torch.empty_like(ud)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=device)
    step_ms, solve_ms = [], []
    with torch.cuda.stream(stream):
        for r in range(reps + 2):
            flush.fill_(r & 0xFF)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            stepper.step(X, u_a, lambda Xs: G, X_out=Xo, u_out=u_b, stream=stream)
            b.record(stream)
            b.synchronize()
            if r >= 2:
                step_ms.append(a.elapsed_time(b))
            X, Xo = Xo, X
            u_a, u_b = u_b, u_a
        f = torch.empty_like(ud).normal_()
        for r in range(reps + 2):
            flush.fill_(r & 0xFF)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            stepper.fluid.solve(f, u_a, rho / dt, mu, u=u_b, stream=stream)
            b.record(stream)
            b.synchronize()
            if r >= 2:
                solve_ms.append(a.elapsed_time(b))
    stepper.plan_n.check(stream)
    stepper.plan_s.check(stream)
    stepper.close()
    solve_bytes = 3 * 3 * N ** 3 * 4
    sm = statistics.mean(solve_ms)
    oracle_ms = None
    if oracle_solve:
        from oracle import stokes as ostokes
        fh = f.double().cpu().numpy()
        uh = u_a.double().cpu().numpy()
        t0 = time.perf_counter()
        ostokes.solve(fh, (N, N, N), (1.0, 1.0, 1.0), rho / dt, mu, uh)
        oracle_ms = (time.perf_counter() - t0) * 1e3
    return {"workload": f"{N}^3 MAC grid, {npts} points, FP32; per step (a) bin + interpolate, (b) advect, "
                        "(d) bin + spread (forces given), (e) Stokes solve (rho 1, mu 0.01, k = bench dt), "
                        "(f) interpolate, (g) advect",
            "step_ms": statistics.mean(step_ms), "pts_per_s": npts / (statistics.mean(step_ms) / 1e3),
            "stokes_solve_ms": sm,
            "oracle_stokes_solve_ms": oracle_ms,
            "oracle_note": "FP64 numpy FFT solve of the same 128^3 MAC problem on the host cores",
            "stokes_roofline": {"bound": "hbm", "achieved_gbs": solve_bytes / (sm / 1e3) / 1e9, "peak": peak,
                                "frac": solve_bytes / (sm / 1e3) / 1e9 / peak, "algorithmic_bytes": solve_bytes,
                                "note": "f, u_old read and u written once; the transforms' own passes not counted"}}


def run_ours(args):
    import torch

    world, rank, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    device = torch.device("cuda", local)
    from paper_2012_06646_gb300 import build
    build()
    from paper_2012_06646_gb300.plan import Plan

    N, npts = args.grid, args.points
    seed = rank_seed(args.seed, rank)
    X0, u = workload(seed, npts, N)
    h = 1.0 / N
    dt = h / (GAMMA * 1.0)            # max |u| = gamma L / 2  ->  max displacement h / 2
    plan = Plan(3, (N, N, N), (1.0, 1.0, 1.0), grid="mac", max_points=npts, device=device)
    stream = torch.cuda.Stream(device)
    nsteps = args.warmup + args.steps
    Gs = [torch.from_numpy(forces(seed, s, npts)).to(device) for s in range(min(nsteps, 16))]
    ud = torch.from_numpy(u).to(device)
    X = torch.from_numpy(X0).to(device)
    f = torch.empty(plan.grid_shape(), dtype=torch.float32, device=device)
    U = torch.empty((npts, 3), dtype=torch.float32, device=device)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=device)
    torch.cuda.synchronize()

    def ev():
        return torch.cuda.Event(enable_timing=True)

    names = ("bin", "interp", "spread", "advect")
    per_call = {k: [] for k in names}
    step_ms = []
    try:
        gpu_id = "GPU-" + str(torch.cuda.get_device_properties(local).uuid)
    except Exception:
        gpu_id = str(local)
    sampler = ClockSampler(gpu_id)
    sampler.start()

    def raw_step(G, e=None):
        if e is not None:
            e[0].record(stream)
        plan.bin(X, stream=stream)
        if e is not None:
            e[1].record(stream)
        plan.interpolate(X, ud, U=U, reuse_bins=True, stream=stream)
        if e is not None:
            e[2].record(stream)
        # interpolation wrote only U: spreading may start during its last wave
        plan.spread(X, G, f=f, reuse_bins=True, overlap_previous=True, stream=stream)
        if e is not None:
            e[3].record(stream)
        plan.advect(X, U, dt, out=X, overlap_previous=True, stream=stream)   # spreading wrote only f
        if e is not None:
            e[4].record(stream)

    # ---- the step as separate calls: per-call times (roofline, breakdown) ----
    plain_ms = []
    with torch.cuda.stream(stream):
        for s in range(nsteps):
            flush.fill_(s & 0xFF)                    # L2 flush, outside the timed events
            e = [ev() for _ in range(5)]
            raw_step(Gs[s % len(Gs)], e)
            if s >= args.warmup:
                e[4].synchronize()
                plain_ms.append(e[0].elapsed_time(e[4]))
                for i, k in enumerate(names):
                    per_call[k].append(e[i].elapsed_time(e[i + 1]))
    torch.cuda.synchronize()

    # ---- the step as one CUDA graph (the same launches, captured once per force
    # buffer so the forces still change every step) ----
    graphs = []
    if not args.no_graph:
        with torch.cuda.stream(stream):
            for G in Gs:
                g = torch.cuda.CUDAGraph()
                with torch.cuda.graph(g, stream=stream):
                    raw_step(G)
                graphs.append(g)
        torch.cuda.synchronize()

    def one_step(s):
        if graphs:
            graphs[s % len(graphs)].replay()
        else:
            raw_step(Gs[s % len(Gs)])

    t_begin = t_end = time.time()
    extra_steps = 0
    with torch.cuda.stream(stream):
        for s in range(nsteps):
            timed = s >= args.warmup
            if timed and s == args.warmup:
                if world > 1:
                    torch.distributed.barrier()
                torch.cuda.synchronize()
                t_begin = time.time()
            flush.fill_(s & 0xFF)                    # L2 flush, outside the timed events
            a, b = ev(), ev()
            a.record(stream)
            one_step(s)
            b.record(stream)
            if timed:
                b.synchronize()
                step_ms.append(a.elapsed_time(b))
        torch.cuda.synchronize()
        try:                                         # outputs of the last timed step, outside the timing
            out_hash = {"f_and_U": output_hash(f, U), "after_steps": nsteps}
        except Exception as exc:
            out_hash = {"error": repr(exc)}
        # nvidia-smi samples every 50 ms: a timed region shorter than that is
        # sampled over a window extended by untimed repeats of the same step.
        while time.time() - t_begin < args.clock_window:
            flush.fill_(extra_steps & 0xFF)
            one_step(nsteps + extra_steps)
            extra_steps += 1
            if extra_steps % 64 == 0:
                torch.cuda.synchronize()
        torch.cuda.synchronize()
        t_end = time.time()
    clocks = sampler.stop(t_begin, t_end)
    if clocks is not None:
        clocks["window_s"] = t_end - t_begin
        clocks["untimed_steps_in_window"] = extra_steps
    plan.check(stream)
    total_ms = max_over_ranks(sum(step_ms), device)
    if world > 1:
        torch.distributed.barrier()
    value = job_rate(npts, world, args.steps, total_ms)

    # ---- end to end through the C ABI with host buffers ----
    e2e = None
    if not args.no_e2e:
        Xh = torch.from_numpy(X0).pin_memory()
        Gh = [g.cpu().pin_memory() for g in Gs[: min(len(Gs), 4)]]
        Uh = torch.empty((npts, 3), dtype=torch.float32).pin_memory()
        fh = torch.empty(plan.grid_shape(), dtype=torch.float32).pin_memory()
        Xd = torch.empty_like(X)
        Xn = torch.empty_like(X)
        Gd = torch.empty_like(Gs[0])
        # Copies overlap the kernels that do not need them, on a copy stream.
        # Interpolation and the position update do not depend on spreading, so
        # the overlapped step runs them first: G uploads during binning and
        # interpolation, U and the new X download while G is spread, and f
        # downloads last; the step ends when both streams are done.
        cs = torch.cuda.Stream(device)

        def sync_ev():
            return torch.cuda.Event()

        e2e_ms, seq_ms = [], []
        with torch.cuda.stream(stream):
            for s in range(2 * nsteps):
                overlapped = s < nsteps
                flush.fill_(s & 0xFF)
                a, b = ev(), ev()
                a.record(stream)
                Xd.copy_(Xh, non_blocking=True)
                if overlapped:
                    # G follows X on the link (binning waits for X only)
                    e_x = sync_ev()
                    e_x.record(stream)
                    cs.wait_event(e_x)
                    with torch.cuda.stream(cs):
                        Gd.copy_(Gh[s % len(Gh)], non_blocking=True)
                    e_g = sync_ev()
                    e_g.record(cs)
                    plan.bin(Xd, stream=stream)
                    plan.interpolate(Xd, ud, U=U, reuse_bins=True, stream=stream)
                    e_in = sync_ev()
                    e_in.record(stream)
                    plan.advect(Xd, U, dt, out=Xn, stream=stream)
                    e_ad = sync_ev()
                    e_ad.record(stream)
                    with torch.cuda.stream(cs):
                        cs.wait_event(e_in)
                        Uh.copy_(U, non_blocking=True)
                        cs.wait_event(e_ad)
                        Xh.copy_(Xn, non_blocking=True)
                    stream.wait_event(e_g)
                    plan.spread(Xd, Gd, f=f, reuse_bins=True, stream=stream)
                    e_sp = sync_ev()
                    e_sp.record(stream)
                    with torch.cuda.stream(cs):
                        cs.wait_event(e_sp)
                        fh.copy_(f, non_blocking=True)
                    e_cs = sync_ev()
                    e_cs.record(cs)
                    stream.wait_event(e_cs)
                else:
                    Gd.copy_(Gh[s % len(Gh)], non_blocking=True)
                    plan.bin(Xd, stream=stream)
                    plan.spread(Xd, Gd, f=f, reuse_bins=True, stream=stream)
                    plan.interpolate(Xd, ud, U=U, reuse_bins=True, stream=stream)
                    plan.advect(Xd, U, dt, out=Xd, stream=stream)
                    Uh.copy_(U, non_blocking=True)
                    fh.copy_(f, non_blocking=True)
                    Xh.copy_(Xd, non_blocking=True)
                b.record(stream)
                b.synchronize()
                if s % nsteps >= args.warmup:
                    (e2e_ms if overlapped else seq_ms).append(a.elapsed_time(b))
        tot = max_over_ranks(sum(e2e_ms), device)
        tot_seq = max_over_ranks(sum(seq_ms), device)

        # Streamed: W + K steps back to back, each step's copies on an upload and a
        # download stream, ordered against the kernels by events only, so step s's
        # downloads run while step s + 1 computes.  Every step still uploads X (the
        # position the previous step wrote back to the host) and G, and downloads U,
        # the new X and f.  Positions and velocity fields are double- and six-fold
        # buffered on the device so no copy waits on a kernel that reads the buffer
        # it would overwrite.
        up_s, dn_s = torch.cuda.Stream(device), torch.cuda.Stream(device)
        Xds = [Xd, torch.empty_like(X)]
        ufields = [ud] + [ud.clone() for _ in range(5)]   # 6 x 25 MB in rotation: more than L2

        def streamed(k_steps: int, s0: int):
            prev, prev2_sp = None, None
            for s in range(k_steps):
                xdb = Xds[s % 2]
                if prev is not None:
                    up_s.wait_event(prev["xdown"])      # Xh holds the previous step's new X
                else:
                    up_s.wait_stream(stream)
                if prev2_sp is not None:
                    up_s.wait_event(prev2_sp)           # the spread that read this X buffer is done
                with torch.cuda.stream(up_s):
                    xdb.copy_(Xh, non_blocking=True)
                e_xup = sync_ev()
                e_xup.record(up_s)
                if prev is not None:
                    up_s.wait_event(prev["sp"])         # the previous spread has read Gd
                with torch.cuda.stream(up_s):
                    Gd.copy_(Gh[(s0 + s) % len(Gh)], non_blocking=True)
                e_g = sync_ev()
                e_g.record(up_s)
                stream.wait_event(e_xup)
                plan.bin(xdb, stream=stream)
                if prev is not None:
                    stream.wait_event(prev["udown"])    # U downloaded before it is overwritten
                plan.interpolate(xdb, ufields[(s0 + s) % len(ufields)], U=U, reuse_bins=True, stream=stream)
                e_in = sync_ev()
                e_in.record(stream)
                plan.advect(xdb, U, dt, out=Xn, stream=stream)
                e_ad = sync_ev()
                e_ad.record(stream)
                dn_s.wait_event(e_ad)
                with torch.cuda.stream(dn_s):
                    Xh.copy_(Xn, non_blocking=True)     # the next step's upload waits for this one
                e_xd = sync_ev()
                e_xd.record(dn_s)
                with torch.cuda.stream(dn_s):
                    Uh.copy_(U, non_blocking=True)
                e_ud = sync_ev()
                e_ud.record(dn_s)
                stream.wait_event(e_g)
                if prev is not None:
                    stream.wait_event(prev["fdown"])    # f downloaded before it is overwritten
                plan.spread(xdb, Gd, f=f, reuse_bins=True, stream=stream)
                e_sp = sync_ev()
                e_sp.record(stream)
                dn_s.wait_event(e_sp)
                with torch.cuda.stream(dn_s):
                    fh.copy_(f, non_blocking=True)
                e_fd = sync_ev()
                e_fd.record(dn_s)
                prev2_sp = prev["sp"] if prev is not None else None
                prev = {"xdown": e_xd, "udown": e_ud, "fdown": e_fd, "sp": e_sp}
            stream.wait_stream(up_s)
            stream.wait_stream(dn_s)

        Xh.copy_(torch.from_numpy(X0))
        with torch.cuda.stream(stream):
            streamed(args.warmup, 0)
            stream.synchronize()
            a, b = ev(), ev()
            a.record(stream)
            streamed(args.steps, args.warmup)
            b.record(stream)
            b.synchronize()
        tot_stream = max_over_ranks(a.elapsed_time(b), device)
        # The streamed results against the same W + K steps run one call after another
        # (outside the timing): equal bit for bit if every copy and kernel kept its order.
        with torch.cuda.stream(stream):
            Xc = torch.from_numpy(X0).to(device)
            Gc = torch.empty_like(Gd)
            for s_ in range(args.warmup + args.steps):
                Gc.copy_(Gh[s_ % len(Gh)])
                plan.bin(Xc, stream=stream)
                Uc = plan.interpolate(Xc, ufields[s_ % len(ufields)], reuse_bins=True, stream=stream)
                Xnc = plan.advect(Xc, Uc, dt, stream=stream)
                fc = plan.spread(Xc, Gc, reuse_bins=True, stream=stream)
                Xc = Xnc
            stream.synchronize()
        streamed_ok = bool(torch.equal(Xh, Xc.cpu()) and torch.equal(Uh, Uc.cpu()) and torch.equal(fh, fc.cpu()))
        e2e = {"value": job_rate(npts, world, args.steps, tot_stream), "unit": "pts/s",
               "h2d_bytes_per_step": int(Xd.numel() * 4 + Gd.numel() * 4),
               "d2h_bytes_per_step": int(Uh.numel() * 4 + fh.numel() * 4 + Xh.numel() * 4),
               "ms_per_step": tot_stream / args.steps,
               "copies": "every step uploads X (the positions the step before wrote back to pinned host memory) and G, "
                         "and downloads U, the new X and f; the K timed steps run back to back, the uploads on one "
                         "stream and the downloads on another, ordered against the kernels by events, so a step's "
                         "downloads overlap the next step's kernels",
               "l2": "no flush inside the streamed window: each step uploads fresh X and G, reads one of six "
                     "velocity fields in rotation (150 MB) and writes 85 MB of tile boxes, more than the 129 MB L2",
               "outputs_equal_sequential": streamed_ok,
               "value_step_by_step": job_rate(npts, world, args.steps, tot),
               "step_by_step": "each step timed alone (L2 flushed before it): X upload on the compute stream; G "
                               "upload after it, during binning and interpolation, U and the new X download while G "
                               "is spread, f download after it (copy stream)",
               "value_copies_serialised": job_rate(npts, world, args.steps, tot_seq)}

    membranes = None
    if args.membrane_reps > 0 and rank == 0:
        try:
            membranes = membrane_bench(device, stream, args.membrane_reps, load_peaks()[0],
                                       oracle_check=not args.no_cpu_baseline)
        except Exception as exc:
            membranes = {"error": repr(exc)}

    paper = None
    if args.paper_reps > 0 and rank == 0:
        try:
            paper = paper_algorithms_bench(plan, X, Gs[0], f, stream, args.paper_reps)
            paper["workload"] = f"{N}^3 MAC grid, {npts} points, FP32, one spread (all three components)"
        except Exception as exc:
            paper = {"error": repr(exc)}

    grad = None
    if args.grad_reps > 0 and rank == 0:
        try:
            grad = autograd_bench(device, stream, args.grad_reps, N)
        except Exception as exc:
            grad = {"error": repr(exc)}

    kern = None
    if args.kernel_reps > 0 and rank == 0:
        try:
            kern = kernels_bench(device, stream, X, Gs[0], ud, args.kernel_reps, N, load_peaks()[0],
                                 0 if args.no_cpu_baseline else 5000)
        except Exception as exc:
            kern = {"error": repr(exc)}

    ibstep = None
    if args.ib_step_reps > 0 and rank == 0:
        try:
            ibstep = ib_step_bench(device, stream, torch.from_numpy(X0).to(device), ud, Gs[0], args.ib_step_reps,
                                   load_peaks()[0], N, dt, oracle_solve=not args.no_cpu_baseline)
        except Exception as exc:
            ibstep = {"error": repr(exc)}

    serving = None
    if args.serve_jobs > 0:
        try:
            serving = serving_bench(device, args.serve_jobs, [float(x) for x in args.serve_loads.split(",")],
                                    world=world, rank=rank)
        except Exception as exc:
            serving = {"error": repr(exc)}

    accuracy = None
    if rank == 0 and not args.no_cpu_baseline:
        try:
            accuracy = accuracy_uniform(plan, X, Gs[0], ud, N, stream, args.seed)
        except Exception as exc:
            accuracy = {"error": repr(exc)}

    if rank != 0:
        if world > 1:
            torch.distributed.destroy_process_group()
        return

    # ---- roofline of the dominant call ----
    peak, peak_kind = load_peaks()
    nc = 3
    alg = {"spread": npts * 3 * 4 + npts * nc * 4 + nc * N ** 3 * 4,
           "interp": npts * 3 * 4 + nc * N ** 3 * 4 + npts * nc * 4}
    mean_ms = {k: statistics.mean(v) for k, v in per_call.items()}
    dom = max(("spread", "interp"), key=lambda k: mean_ms[k])
    achieved = alg[dom] / (mean_ms[dom] / 1e3) / 1e9
    traffic = ncu_traffic(dom)
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": traffic, "kernel": dom, "peak_source": f"{peak_kind} hbm_gbs (copy)",
                "algorithmic_bytes_per_launch": alg[dom]}

    cpu = cpu_all = None
    if not args.no_cpu_baseline:
        try:
            import oracle
            oracle.build()
            rate, secs = cpu_oracle_rate(min(args.cpu_sample, npts), N, args.seed)
            cpu = {"value": rate, "unit": "pts/s", "cores": 1, "kind": "oracle",
                   "sample": f"{min(args.cpu_sample, npts)} of the {npts} points, one FP64 spread + one "
                             f"interpolation on the {N}^3 MAC grid, single thread ({secs:.1f} s)"}
        except Exception as exc:  # the baseline is reported, never required
            cpu = {"value": None, "unit": "pts/s", "cores": 1, "kind": "oracle", "sample": f"failed: {exc}"}
        try:
            rate, secs, procs = cpu_oracle_parallel(N, args.seed, npts)
            cpu_all = {"value": rate, "unit": "pts/s", "cores": procs, "kind": "oracle",
                       "sample": f"all {npts} points, one FP64 spread + one interpolation on the {N}^3 MAC grid, "
                                 f"split over {procs} processes (per-process grids summed in order; {secs:.1f} s)"}
        except Exception as exc:
            cpu_all = {"value": None, "unit": "pts/s", "cores": None, "kind": "oracle", "sample": f"failed: {exc}"}


    launches_per_step = 4 + 2 + 1 + 1     # bin: count, scan, scatter, stable; spread: tile boxes, combine;
    #                                        interp: tiles (+ invalid points); advect
    line = {"metric": METRIC, "value": value, "unit": "pts/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"{N}^3 MAC grid, {npts} uniform points per GPU, FP32, standard 4-point "
                                   "kernel; per step: bin, interpolate, spread (overlapping the interpolation's tail), advect",
                       "grid": N, "n_points": npts, "steps": args.steps,
                       "l2": "flushed between timed steps (256 MB write)", "parallelism": f"replicas x{world}"},
            "roofline": roofline, "cpu_baseline": cpu, "cpu_baseline_all_cores": cpu_all, "e2e": e2e,
            "gpu_launches": launches_per_step * args.steps,
            "clocks": clocks,
            "calls_ms": mean_ms,
            "step_ms_as_separate_calls": statistics.mean(plain_ms) if plain_ms else None,
            "step_as_cuda_graph": bool(graphs),
            "step_ms_distribution": step_distribution(step_ms),
            "calls_ms_distribution": {k: step_distribution(v) for k, v in per_call.items()},
            "output_sha256_16": out_hash,
            "error_vs_fp64_oracle": accuracy,
            "serving": serving,
            "membranes": membranes,
            "paper_algorithms": paper,
            "differentiable": grad,
            "kernel_widths": kern,
            "ib_step": ibstep}
    print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
