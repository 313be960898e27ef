"""Host logic of the z-slab decomposition (paper_2012_06646_gb300/slab.py), on
CPU: the layer split and the periodic neighbours; and, on two and three gloo
ranks, the halo exchange (each rank's recv_lo is its lower neighbour's
send_hi, recv_hi its upper neighbour's send_lo), the field-plane halo that
interpolation needs, and the routing of points to the rank of their slab and
of per-point results back.  Cell indices of the routing come from the FP64
oracle's cell map, the same exact map ib_slab_owner uses on the GPU."""
import os
import socket
import sys

import numpy as np
import pytest
import torch
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_layer_bounds_and_neighbours():
    from paper_2012_06646_gb300 import slab
    assert slab.layer_bounds(16, 2) == [0, 8, 16]
    assert slab.layer_bounds(6, 4) == [0, 2, 4, 5, 6]
    assert slab.layer_bounds(5, 5) == [0, 1, 2, 3, 4, 5]
    with pytest.raises(ValueError):
        slab.layer_bounds(3, 4)
    assert slab.neighbours(0, 3) == (2, 1) and slab.neighbours(2, 3) == (1, 0)
    assert slab.neighbours(0, 1) == (0, 0)


def test_field_halo_planes_on_one_process():
    """Three slabs of a 48-plane field: each slab's array ends up with its own planes plus two
    planes from each neighbour (periodic), and nothing else."""
    from paper_2012_06646_gb300 import slab
    nz = 48
    u = torch.arange(2 * nz * 2 * 3, dtype=torch.float64).reshape(2, nz, 2, 3)
    bounds = slab.layer_bounds(nz // 8, 3)
    fields = []
    for k in range(3):
        v = torch.full_like(u, float("nan"))
        z0, z1 = 8 * bounds[k], 8 * bounds[k + 1]
        v[:, z0:z1] = u[:, z0:z1]
        fields.append(v)
    sends = [slab.field_sends(v, bounds[k], bounds[k + 1]) for k, v in enumerate(fields)]
    for k, v in enumerate(fields):
        lo, hi = slab.neighbours(k, 3)
        slab.field_receive(v, bounds[k], bounds[k + 1], sends[lo][1], sends[hi][0])
    for k, v in enumerate(fields):
        z0, z1 = 8 * bounds[k], 8 * bounds[k + 1]
        want = {z % nz for z in range(z0 - 2, z1 + 2)}
        for z in range(nz):
            if z in want:
                assert torch.equal(v[:, z], u[:, z])
            else:
                assert bool(torch.isnan(v[:, z]).all())


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import ib_inputs
        import oracle
        from paper_2012_06646_gb300 import slab
        res = {}
        # box planes: send_lo / send_hi tagged with (rank, side)
        send_lo = torch.full((1000,), 10.0 * rank + 1)
        send_hi = torch.full((1000,), 10.0 * rank + 2)
        recv_lo, recv_hi = torch.empty(1000), torch.empty(1000)
        slab.exchange_dist(send_lo, send_hi, recv_lo, recv_hi, rank, world)
        lo, hi = slab.neighbours(rank, world)
        res["boxes"] = bool(torch.all(recv_lo == 10.0 * lo + 2)) and bool(torch.all(recv_hi == 10.0 * hi + 1))
        # field halo: the neighbours' planes, exchanged as contiguous plane blocks
        nz, bounds = 32, slab.layer_bounds(4, world)
        u = torch.arange(3 * nz * 4 * 5, dtype=torch.float64).reshape(3, nz, 4, 5)
        zb, ze = bounds[rank], bounds[rank + 1]
        mine = torch.full_like(u, float("nan"))
        mine[:, 8 * zb:8 * ze] = u[:, 8 * zb:8 * ze]
        to_lo, to_hi = (t.contiguous() for t in slab.field_sends(mine, zb, ze))
        from_lo, from_hi = torch.empty_like(to_hi), torch.empty_like(to_lo)
        slab.exchange_dist(to_lo, to_hi, from_lo, from_hi, rank, world)
        slab.field_receive(mine, zb, ze, from_lo, from_hi)
        ok = True
        for z in range(8 * zb - 2, 8 * ze + 2):
            ok = ok and bool(torch.equal(mine[:, z % nz], u[:, z % nz]))
        res["field"] = ok
        # routing: every rank starts with its own arbitrary share of the points
        n, L = (16, 16, 32), (1.0, 1.0, 1.0)
        X = ib_inputs.uniform_points(40 + rank, 500, L, 3)
        X[::50] = np.nan                                               # invalid positions stay unrouted
        g = oracle.Grid(dim=3, n=n, L=L)
        ok_pts = ~np.isnan(X).any(axis=1)
        cz = np.full(len(X), -1)
        cz[ok_pts] = (oracle.cell_keys(g, X[ok_pts].astype(np.float64)) // (16 * 16)).astype(np.int64)
        owner = np.where(cz >= 0, np.searchsorted(np.array(bounds) * 8, np.maximum(cz, 0), side="right") - 1, -1)
        idx = torch.arange(len(X), dtype=torch.int64) + 1000 * rank      # global point ids
        (Xr, idr), info = slab.route_points(torch.from_numpy(owner), [torch.from_numpy(X), idx], rank, world)
        czr = (oracle.cell_keys(g, Xr.numpy().astype(np.float64)) // (16 * 16)).astype(np.int64)
        res["route_owned"] = bool(np.all((czr >= 8 * zb) & (czr < 8 * ze)))
        res["route_count"] = int(len(Xr))
        res["route_valid_sent"] = int(ok_pts.sum())
        # results back: each owner returns its points' ids, which must come back in place
        back = slab.route_back(idr.to(torch.float64)[:, None], info, len(X))
        res["route_back"] = bool(np.array_equal(back[ok_pts, 0].numpy(), idx[ok_pts].numpy().astype(np.float64))) \
            and bool(torch.isnan(back[~torch.from_numpy(ok_pts), 0]).all())
        out.put((rank, res))
        dist.barrier()
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_exchange_and_routing_on_gloo_ranks(world):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=180) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r in range(world):
        assert res[r]["boxes"] and res[r]["field"] and res[r]["route_owned"] and res[r]["route_back"], res[r]
    assert sum(res[r]["route_count"] for r in range(world)) == sum(res[r]["route_valid_sent"] for r in range(world))
