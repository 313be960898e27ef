"""Served form: a persistent request loop with continuous batching.

Each request is one independent job: a periodic 3-D MAC grid of its own size
and a point set of its own size; the job spreads its forces onto its grid
and interpolates that grid back to its points (f = S G, U = S* f; the grid
never leaves the device).  The loop

  * admits waiting requests into a wave whenever one of `nstreams` wave
    slots is free, as long as the wave fits the slot's batch capacity and
    the in-flight HBM footprint (I/O buffers + scratch share) fits the
    budget -- requests that arrive while other waves run on the GPU join
    the next free slot, so their work overlaps on the device;
  * runs a wave as one ib_batch_run_host call: the jobs' inputs are copied
    from pinned host memory into the slot's device buffers, the wave runs
    in a fixed number of launches for any number of jobs, and U is copied
    back, all on the slot's stream;
  * retires a wave when its completion event fires, reads the copy of the
    device error word that the wave's own stream left in pinned memory (the
    blocking read-and-clear on the slot's stream only when it shows an error)
    and records each request's outcome and latency (completion minus arrival).

Failures are handled on the host, per request: a job that can never fit a
wave slot (points, cells or tiles above the slot's capacity, or an invalid
grid) is rejected when it arrives instead of waiting forever; a request whose
`cancelled` flag is set before admission is dropped, and one cancelled while
its wave runs finishes on the device but is reported as cancelled; a wave
whose error word reports non-finite or out-of-range positions marks the
requests whose results carry NaN (the kernels' output for such points) as
invalid and the others as done.  If the arena of a wave slot after the first
cannot be allocated (IB_ERR_OOM), the server runs with the slots it has.

`single_job_loop` is the comparison: per job, copy in, ib_spread +
ib_interpolate on a plan for its grid size, copy U out, wait.
A job's result is the same whether it runs alone or in a mix: the batched
kernels give each job its own bins, tiles and summation order.
"""

from __future__ import annotations

import collections
import gc
import time
from dataclasses import dataclass, field

import numpy as np
import torch

from . import _abi
from ._abi import IBError
from .plan import Batch, Plan

# Outcomes of a request (Request.status).
WAITING, DONE, REJECTED, CANCELLED, INVALID = "waiting", "done", "rejected", "cancelled", "invalid_positions"


@dataclass
class Request:
    rid: int
    N: int
    X: torch.Tensor                  # (n, 3) float32, pinned host
    G: torch.Tensor                  # (n, 3) float32, pinned host
    arrival: float = 0.0             # seconds from the start of serving
    L: float = 1.0
    U: torch.Tensor | None = None    # result, pinned host
    t_admit: float = -1.0
    t_done: float = -1.0
    cancelled: bool = False          # set by the caller (Server.cancel) at any time
    status: str = WAITING            # outcome once served: done, rejected, cancelled, invalid_positions
    reason: str = ""                 # why a request was rejected

    @property
    def npts(self) -> int:
        return int(self.X.shape[0])

    def io_bytes(self) -> int:
        return int(self.npts * 3 * 4 * 3 + 3 * self.N ** 3 * 4)


@dataclass
class _Wave:
    reqs: list
    bufs: list
    event: torch.cuda.Event
    footprint: int


@dataclass
class ServeStats:
    latencies_ms: list = field(default_factory=list)
    wall_s: float = 0.0
    points: int = 0
    jobs: int = 0
    waves: int = 0
    max_inflight_bytes: int = 0
    outcomes: dict = field(default_factory=dict)

    def summary(self) -> dict:
        lat = np.array(self.latencies_ms) if self.latencies_ms else np.zeros(1)
        return {"jobs": self.jobs, "waves": self.waves, "wall_s": self.wall_s, "outcomes": dict(self.outcomes),
                "pts_per_s": self.points / self.wall_s if self.wall_s > 0 else None,
                "jobs_per_s": self.jobs / self.wall_s if self.wall_s > 0 else None,
                "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
                "mean_ms": float(lat.mean()), "max_inflight_bytes": self.max_inflight_bytes}


@dataclass
class WaveCaps:
    jobs: int
    points: int
    cells: int
    tiles: int


def place_jobs(costs, world: int) -> list:
    """Owner rank of each job when a batch of independent jobs is sharded over `world` GPUs
    (no collective: each rank serves its own jobs).  Longest job first onto the rank with the
    least work so far (ties: the lower rank), so the ranks' loads differ by at most one job's
    cost; deterministic, so every rank computes the same placement.  costs: work per job (for
    a spread + interpolate job, its points plus its grid cells)."""
    if world < 1:
        raise ValueError("world must be >= 1")
    order = sorted(range(len(costs)), key=lambda i: (-costs[i], i))
    load = [0] * world
    owner = [0] * len(costs)
    for i in order:
        r = min(range(world), key=lambda k: (load[k], k))
        owner[i] = r
        load[r] += costs[i]
    return owner


def never_fits(npts: int, cells: int, tiles: int, caps: WaveCaps) -> str:
    """Why a job can never join a wave of a slot with capacities `caps` ('' if it can)."""
    if npts > caps.points:
        return f"{npts} points exceed the slot's {caps.points}"
    if cells > caps.cells:
        return f"{cells} grid cells exceed the slot's {caps.cells}"
    if tiles > caps.tiles:
        return f"{tiles} spreading tiles exceed the slot's {caps.tiles}"
    return ""


def admit_wave(queue, caps: WaveCaps, inflight: int, budget: int):
    """FIFO admission of waiting jobs into one wave.

    queue: (npts, cells, footprint_bytes, tiles) per waiting job, in arrival order.
    A job joins while the wave stays within the slot's capacity and the
    in-flight footprint stays within the HBM budget; a job larger than the
    whole budget still runs when nothing else is in flight (else it would
    wait forever).  Returns (number of jobs admitted, wave footprint).
    """
    n, fp, pts, cells, tiles = 0, 0, 0, 0, 0
    for npts, ncell, rf, rt in queue:
        if n >= caps.jobs or pts + npts > caps.points or cells + ncell > caps.cells or tiles + rt > caps.tiles:
            break
        if inflight + fp + rf > budget and (n > 0 or inflight > 0):
            break
        n += 1
        fp += rf
        pts += npts
        cells += ncell
        tiles += rt
    return n, fp


class Server:
    def __init__(self, nstreams: int = 3, max_jobs: int = 256, max_points: int = 1 << 23,
                 max_cells: int = 1 << 26, budget_bytes: int | None = None, device=None):
        self.device = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        self.batches, self.streams = [], []
        for k in range(nstreams):
            try:
                b = Batch(dim=3, grid="mac", max_jobs=max_jobs, max_points=max_points, max_cells=max_cells,
                          max_tiles=max_cells // 512 + 8 * max_jobs, host_io=True, device=self.device)
            except IBError as e:
                if e.status != _abi.IB_ERR_OOM or k == 0:
                    raise
                break                   # run with the slots that could be allocated
            self.batches.append(b)
            self.streams.append(torch.cuda.Stream(self.device))
        self.nstreams = len(self.batches)
        self.cap = (max_jobs, max_points, max_cells)
        if budget_bytes is None:
            free, _ = torch.cuda.mem_get_info(self.device)
            budget_bytes = int(0.5 * free)
        self.budget = int(budget_bytes)

    def cancel(self, r: Request) -> None:
        """Cancel a request: dropped if not yet admitted, else reported as cancelled when its wave ends."""
        r.cancelled = True

    def caps(self, slot: int = 0) -> WaveCaps:
        return WaveCaps(self.cap[0], self.cap[1], self.cap[2], self.batches[slot].desc.max_tiles)

    def footprint(self, r: Request) -> tuple:
        job = self.batches[0].job_struct((r.N, r.N, r.N), (r.L, r.L, r.L), r.X)
        scratch, tiles = self.batches[0].job_footprint(job)
        return r.io_bytes() + scratch, tiles

    def _launch(self, slot: int, reqs: list, footprint: int) -> _Wave:
        s = self.streams[slot]
        for r in reqs:
            if r.U is None:
                r.U = torch.empty((r.npts, 3), dtype=torch.float32).pin_memory()
        self.batches[slot].run_host([((r.N, r.N, r.N), (r.L, r.L, r.L), r.X, r.G, r.U) for r in reqs], stream=s)
        ev = torch.cuda.Event()
        ev.record(s)
        return _Wave(reqs=reqs, bufs=[], event=ev, footprint=footprint)

    def serve(self, requests: list, realtime: bool = True) -> ServeStats:
        """Serve `requests` (sorted by arrival).  realtime=False admits everything at t = 0.
        Python's cyclic garbage collector is paused while the loop runs: a collection over
        thousands of live request objects can stall it for tens of milliseconds."""
        with _gc_paused():
            return self._serve(requests, realtime)

    def _serve(self, requests: list, realtime: bool) -> ServeStats:
        stats = StatsAccumulator()
        pending = collections.deque(sorted(requests, key=lambda r: r.arrival))
        waiting: collections.deque = collections.deque()
        slots: list = [None] * self.nstreams
        inflight = 0
        t0 = time.perf_counter()
        sizes = {}
        caps0 = self.caps(0)
        while pending or waiting or any(w is not None for w in slots):
            now = time.perf_counter() - t0
            while pending and (not realtime or pending[0].arrival <= now):
                r = pending.popleft()
                try:
                    sizes[r.rid] = self.footprint(r)
                    r.reason = never_fits(r.npts, r.N ** 3, sizes[r.rid][1], caps0)
                except IBError as e:          # invalid job description
                    r.reason = str(e)
                if r.reason:
                    r.status = REJECTED
                    r.t_done = time.perf_counter() - t0
                    stats.add(r)
                else:
                    waiting.append(r)
            for i, w in enumerate(slots):
                if w is not None and w.event.query():
                    tdone = time.perf_counter() - t0
                    # the wave's copy of the error word; the blocking read-and-clear only on an error
                    err = self.batches[i].wave_status()
                    if err != _abi.IB_OK:
                        err = self.batches[i].status(self.streams[i])
                    if err not in (_abi.IB_OK, _abi.IB_ERR_NONFINITE, _abi.IB_ERR_RANGE):
                        raise IBError(err, "served wave")
                    for r in w.reqs:
                        r.t_done = tdone
                        if r.cancelled:
                            r.status = CANCELLED
                        elif err != _abi.IB_OK and not bool(torch.isfinite(r.U).all()):
                            r.status = INVALID
                        else:
                            r.status = DONE
                        stats.add(r)
                    inflight -= w.footprint
                    slots[i] = None
            if any(r.cancelled for r in waiting):
                keep = collections.deque()
                for r in waiting:
                    if r.cancelled:
                        r.status = CANCELLED
                        r.t_done = time.perf_counter() - t0
                        stats.add(r)
                    else:
                        keep.append(r)
                waiting = keep
            for i in range(self.nstreams):
                if slots[i] is not None or not waiting:
                    continue
                caps = self.caps(i)
                take, fp = admit_wave([(r.npts, r.N ** 3) + sizes[r.rid] for r in waiting], caps, inflight,
                                      self.budget)
                wave = [waiting.popleft() for _ in range(take)]
                for r in wave:
                    r.t_admit = time.perf_counter() - t0
                if wave:
                    slots[i] = self._launch(i, wave, fp)
                    inflight += fp
                    stats.waves += 1
                    stats.max_inflight = max(stats.max_inflight, inflight)
            if realtime and not waiting and pending and all(w is None for w in slots):
                # Idle until the next arrival: sleep only through a gap longer than 50 ms
                # (waking 10 ms early), spin otherwise.  A sleep overshoots by tens of
                # microseconds, and by milliseconds when the core drops into a deep idle
                # state; a spinning loop reacts at once, as the single-job loop it is
                # compared with does.
                target = pending[0].arrival
                delay = target - (time.perf_counter() - t0)
                if delay > 0.05:
                    time.sleep(delay - 0.01)
                while time.perf_counter() - t0 < target:
                    pass
        torch.cuda.synchronize(self.device)
        for b in self.batches:
            b.check()
        return stats.finish(time.perf_counter() - t0)

    def close(self):
        for b in self.batches:
            b.close()


class StatsAccumulator:
    def __init__(self):
        self.lat = []
        self.points = 0
        self.jobs = 0
        self.waves = 0
        self.max_inflight = 0
        self.outcomes = {}

    def add(self, r: Request):
        """Count a finished request; latency and throughput count completed jobs only."""
        if r.status == WAITING:
            r.status = DONE
        self.outcomes[r.status] = self.outcomes.get(r.status, 0) + 1
        if r.status != DONE:
            return
        self.lat.append(1e3 * (r.t_done - r.arrival))
        self.points += r.npts
        self.jobs += 1

    def finish(self, wall: float) -> ServeStats:
        return ServeStats(latencies_ms=self.lat, wall_s=wall, points=self.points, jobs=self.jobs, waves=self.waves,
                          max_inflight_bytes=self.max_inflight, outcomes=dict(self.outcomes))


class _gc_paused:
    """Pause the cyclic garbage collector for the duration of a serving loop."""

    def __enter__(self):
        self.was = gc.isenabled()
        gc.disable()

    def __exit__(self, *exc):
        if self.was:
            gc.enable()


def single_job_loop(requests: list, realtime: bool = True, device=None) -> ServeStats:
    """One job per launch sequence: for each request in arrival order, copy X and G in, ib_spread +
    ib_interpolate on a plan for its grid size, copy U out, wait (the garbage collector paused, as
    for the server)."""
    with _gc_paused():
        return _single_job_loop(requests, realtime, device)


def _single_job_loop(requests: list, realtime: bool, device) -> ServeStats:
    device = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
    plans, bufs = {}, {}
    maxn = collections.defaultdict(int)
    for r in requests:
        maxn[r.N] = max(maxn[r.N], r.npts)
    for N, m in maxn.items():
        plans[N] = Plan(3, (N, N, N), (1.0, 1.0, 1.0), grid="mac", max_points=m, device=device)
        bufs[N] = (torch.empty((m, 3), dtype=torch.float32, device=device),
                   torch.empty((m, 3), dtype=torch.float32, device=device),
                   torch.empty((m, 3), dtype=torch.float32, device=device),
                   torch.empty((3, N, N, N), dtype=torch.float32, device=device))
    for r in requests:
        if r.U is None:
            r.U = torch.empty((r.npts, 3), dtype=torch.float32).pin_memory()
    stats = StatsAccumulator()
    s = torch.cuda.Stream(device)
    order = sorted(requests, key=lambda r: r.arrival)
    t0 = time.perf_counter()
    with torch.cuda.stream(s):
        for r in order:
            if realtime:
                while time.perf_counter() - t0 < r.arrival:
                    pass
            p = plans[r.N]
            Xb, Gb, Ub, f = bufs[r.N]
            X, G, U = Xb[: r.npts], Gb[: r.npts], Ub[: r.npts]
            X.copy_(r.X, non_blocking=True)
            G.copy_(r.G, non_blocking=True)
            p.spread(X, G, f=f, stream=s)
            p.interpolate(X, f, U=U, reuse_bins=True, stream=s)
            r.U.copy_(U, non_blocking=True)
            s.synchronize()
            r.t_done = time.perf_counter() - t0
            stats.add(r)
    for p in plans.values():
        p.check(s)
        p.close()
    return stats.finish(time.perf_counter() - t0)


def make_requests(specs, L: float = 1.0, arrivals=None) -> list:
    """Requests from ib_inputs job specs (positions and N(0,1) forces), pinned host buffers."""
    import ib_inputs
    out = []
    for i, sp in enumerate(specs):
        X = ib_inputs.job_points(sp, L)
        G = ib_inputs.normal_array(sp.seed, (sp.npts, 3), purpose="job-G")
        out.append(Request(rid=i, N=sp.N, X=torch.from_numpy(X).pin_memory(), G=torch.from_numpy(G).pin_memory(),
                           arrival=float(arrivals[i]) if arrivals is not None else 0.0, L=L,
                           U=torch.empty((sp.npts, 3), dtype=torch.float32).pin_memory()))
    return out
