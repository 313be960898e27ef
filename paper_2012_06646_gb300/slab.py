"""z-slab decomposition of one spread + interpolate problem (multi-GPU prototype).

The grid is cut along z into slabs of whole 8-node tile layers; slab k owns
layers [b_k, b_{k+1}), the node planes [8 b_k, 8 b_{k+1}) and the points
whose cell lies in them (ib_slab_owner).  Spreading: each slab forms the tile
boxes of its layers (ib_slab_spread) and sends the box planes that reach
past its ends -- two node planes each side -- to its neighbours, which place
them and form f on their own planes (ib_slab_combine); the result equals the
single-plan spread bit for bit.  Interpolation: each slab receives two node
planes of the field from each neighbour (a halo copy) and interpolates its
own points with ib_interpolate.  The exchange is a copy between neighbours
(periodic in z): `exchange_local` for slabs held by one process (one GPU),
`exchange_dist` for one slab per rank over torch.distributed point-to-point
messages.  `route_points` / `route_back` move points to the rank of their slab and
results back (all-to-all).  Everything computed here is index bookkeeping
and data movement; the method's arithmetic runs in the library's kernels.
"""

from __future__ import annotations

import ctypes

import torch

from . import _abi
from ._abi import check
from .plan import Plan, _ptr, _stream_ptr

TILE = 8        # node planes per tile layer along z
HALO = 2        # node planes a slab needs beyond each of its ends


def layer_bounds(nlayers: int, nslab: int) -> list:
    """Balanced split of nlayers tile layers into nslab slabs: [b_0 = 0, ..., b_nslab = nlayers]."""
    if nslab < 1 or nslab > nlayers:
        raise ValueError(f"cannot split {nlayers} tile layers into {nslab} slabs")
    q, r = divmod(nlayers, nslab)
    b = [0]
    for k in range(nslab):
        b.append(b[-1] + q + (1 if k < r else 0))
    return b


def neighbours(k: int, nslab: int) -> tuple:
    """(lower, upper) neighbour slabs of slab k, periodic in z."""
    return (k - 1) % nslab, (k + 1) % nslab


def owners(plan: Plan, X, bounds, stream=None) -> torch.Tensor:
    """Slab of each point (int32; -1 for an invalid position), from the exact cell map."""
    n = plan._points(X)
    out = torch.empty(n, dtype=torch.int32, device=plan.device)
    arr = (ctypes.c_int * len(bounds))(*[int(v) for v in bounds])
    check(plan.lib.ib_slab_owner(plan.handle, n, _ptr(X), len(bounds) - 1, arr, _ptr(out), _stream_ptr(stream)),
          "ib_slab_owner")
    return out


class Slab:
    """Slab k of a z-split of plan's grid: its layers, its halo buffers and its calls."""

    def __init__(self, plan: Plan, k: int, bounds, compensated: bool = False):
        self.plan, self.k, self.bounds = plan, k, list(bounds)
        self.zb, self.ze = self.bounds[k], self.bounds[k + 1]
        self.nslab = len(self.bounds) - 1
        self.flags = _abi.IB_COMPENSATED if compensated else 0
        nbytes = ctypes.c_size_t()
        check(plan.lib.ib_slab_halo_bytes(plan.handle, self.flags, ctypes.byref(nbytes)), "ib_slab_halo_bytes")
        self.halo_bytes = int(nbytes.value)
        mk = lambda: torch.empty(self.halo_bytes, dtype=torch.uint8, device=plan.device)  # noqa: E731
        self.send_lo, self.send_hi, self.recv_lo, self.recv_hi = mk(), mk(), mk(), mk()

    @property
    def planes(self) -> tuple:
        """Node planes [z0, z1) this slab owns."""
        return TILE * self.zb, TILE * self.ze

    def spread(self, X, G, reuse_bins: bool = False, stream=None) -> None:
        """Boxes of the slab's layers from its points, and the planes for the neighbours (send_lo, send_hi)."""
        p = self.plan
        n = p._points(X)
        p._check(G, (n, p.ncomp), "G")
        flags = self.flags | (_abi.IB_REUSE_BINS if reuse_bins else 0)
        if not reuse_bins:
            p.bin_epoch += 1
        check(p.lib.ib_slab_spread(p.handle, n, _ptr(X), _ptr(G), self.zb, self.ze, _ptr(self.send_lo),
                                   _ptr(self.send_hi), flags, _stream_ptr(stream)), "ib_slab_spread")

    def combine(self, f, accumulate: bool = False, stream=None) -> None:
        """f on the slab's own planes, from its boxes and the received planes (recv_lo, recv_hi)."""
        p = self.plan
        p._check(f, p.grid_shape(), "f")
        flags = self.flags | (_abi.IB_ACCUMULATE if accumulate else 0)
        check(p.lib.ib_slab_combine(p.handle, _ptr(f), self.zb, self.ze, _ptr(self.recv_lo), _ptr(self.recv_hi),
                                    flags, _stream_ptr(stream)), "ib_slab_combine")

    # ---- interpolation halo: node planes of the field ----
    def field_sends(self, u) -> tuple:
        return field_sends(u, self.zb, self.ze)

    def field_receive(self, u, from_lower, from_upper) -> None:
        field_receive(u, self.zb, self.ze, from_lower, from_upper)


def field_sends(u, zb: int, ze: int) -> tuple:
    """The field planes a slab of layers [zb, ze) sends: HALO planes to its lower neighbour (its first
    ones) and HALO to its upper neighbour (its last ones); u is [ncomp][nz][ny][nx]."""
    z0, z1 = TILE * zb, TILE * ze
    return u[:, z0:z0 + HALO], u[:, z1 - HALO:z1]


def field_receive(u, zb: int, ze: int, from_lower, from_upper) -> None:
    """Place the neighbours' planes in the slab's array: HALO planes below the slab and HALO above it
    (node planes wrap periodically)."""
    nz = u.shape[1]
    z0, z1 = TILE * zb, TILE * ze
    for i in range(HALO):
        u[:, (z0 - HALO + i) % nz].copy_(from_lower[:, i])
        u[:, (z1 + i) % nz].copy_(from_upper[:, i])


def exchange_local(slabs: list) -> None:
    """Box planes between the slabs of one process: recv_lo of slab k = send_hi of its lower
    neighbour, recv_hi = send_lo of its upper neighbour."""
    n = len(slabs)
    for k, s in enumerate(slabs):
        lo, hi = neighbours(k, n)
        s.recv_lo.copy_(slabs[lo].send_hi)
        s.recv_hi.copy_(slabs[hi].send_lo)


def exchange_field_local(slabs: list, fields: list) -> None:
    """Field halo between the slabs of one process: each slab's array gets HALO planes from each neighbour."""
    n = len(slabs)
    sends = [s.field_sends(u) for s, u in zip(slabs, fields)]
    for k, (s, u) in enumerate(zip(slabs, fields)):
        lo, hi = neighbours(k, n)
        s.field_receive(u, sends[lo][1], sends[hi][0])


def exchange_dist(send_lo, send_hi, recv_lo, recv_hi, rank: int, world: int, group=None) -> None:
    """One slab per rank: send_lo to the lower neighbour (its recv_hi), send_hi to the upper one (its
    recv_lo), over torch.distributed point-to-point messages (NCCL between GPUs, gloo on the host);
    periodic, so with two ranks both messages go to the same peer (told apart by their tags)."""
    import torch.distributed as dist
    lo, hi = neighbours(rank, world)
    if world == 1:
        recv_lo.copy_(send_hi)
        recv_hi.copy_(send_lo)
        return
    # messages to one peer are matched in posting order (and by tag where the backend has tags)
    reqs = [dist.irecv(recv_hi, hi, group=group, tag=0), dist.irecv(recv_lo, lo, group=group, tag=1),
            dist.isend(send_lo, lo, group=group, tag=0), dist.isend(send_hi, hi, group=group, tag=1)]
    for req in reqs:
        req.wait()


def route_points(owner, tensors, rank: int, world: int, group=None) -> tuple:
    """Send every point to the rank that owns its slab (torch.distributed all-to-all): owner (n,)
    int32/int64 on this rank, tensors a list of (n, c) arrays of the same points (positions, forces,
    indices ...).  Returns the received rows of each tensor (points of this rank's slab, grouped by
    source rank, each group in its source order) and the per-source counts, which `route_back` uses
    to return per-point results.  Points with owner -1 (invalid positions) stay with no rank."""
    import torch.distributed as dist
    owner = owner.to(torch.int64)
    order = torch.argsort(owner, stable=True)
    send_counts = torch.bincount(owner[owner >= 0], minlength=world)[:world].to(torch.int64)
    keep = order[(owner[order] >= 0)]
    recv_counts = torch.empty_like(send_counts)
    dist.all_to_all_single(recv_counts, send_counts, group=group)
    out = []
    for t in tensors:
        src = t[keep].contiguous()
        dst = torch.empty((int(recv_counts.sum()),) + tuple(t.shape[1:]), dtype=t.dtype, device=t.device)
        dist.all_to_all_single(dst, src, recv_counts.tolist(), send_counts.tolist(), group=group)
        out.append(dst)
    return out, (send_counts, recv_counts, keep)


def route_back(result, plan_info, n: int, fill=float("nan"), group=None):
    """Return per-point results computed by the owners to the ranks the points came from, in their
    original order (rows of points with no owner get `fill`)."""
    import torch.distributed as dist
    send_counts, recv_counts, keep = plan_info
    back = torch.empty((int(send_counts.sum()),) + tuple(result.shape[1:]), dtype=result.dtype, device=result.device)
    dist.all_to_all_single(back, result.contiguous(), send_counts.tolist(), recv_counts.tolist(), group=group)
    out = torch.full((n,) + tuple(result.shape[1:]), fill, dtype=result.dtype, device=result.device)
    out[keep] = back
    return out
