"""Cases run twice by test_gpu_debug_bounds.py: once on the release library and
once, in a child process, on the IB_DEBUG_BOUNDS build.  Each case runs
through the public binding, checks the plan's error word (the debug build
reports a failed index check there as IB_ERR_BOUNDS) and returns a SHA-256
of its outputs, so the two builds can be compared bit for bit.

The cases cover the kernel families and their edge paths: 3-D and 2-D, MAC
and cell-centred, FP32 and FP64, the three-component and per-component
spreading kernels, grids below the fast-combine size and with ragged last
tiles, points on the periodic seam, clustered points (empty tiles skipped),
compensated and accumulating spreading, position gradients, the 3- and
6-point kernels, walls, and a batched wave."""
import hashlib
import json
import sys

import numpy as np
import torch


def _h(*ts) -> str:
    m = hashlib.sha256()
    for t in ts:
        m.update(np.ascontiguousarray(t.detach().cpu().numpy()).tobytes())
    return m.hexdigest()


def _pts(seed, n, dim, dtype, lo=0.0, hi=1.0, seam=False):
    g = np.random.default_rng(seed)
    X = lo + (hi - lo) * g.random((n, dim))
    if seam:                                   # a fifth of the points within 1e-3 of a periodic face
        k = n // 5
        X[:k, 0] = np.where(g.random(k) < 0.5, 1e-4 * g.random(k), 1.0 - 1e-4 * g.random(k))
    return torch.from_numpy(X).to(dtype).cuda()


def run_cases() -> dict:
    from paper_2012_06646_gb300 import _abi
    from paper_2012_06646_gb300.plan import Batch, Plan
    out = {"version": _abi.load().ib_version().decode()}
    specs = [
        # name, dim, n, grid, kernel, dtype, ncomp, npts, extra
        ("mac3_f32", 3, (48, 40, 32), "mac", "peskin4", torch.float32, None, 20000, {"seam": True}),
        ("mac3_f64", 3, (16, 16, 16), "mac", "peskin4", torch.float64, None, 600, {}),
        ("cc3_f32_c1", 3, (24, 24, 24), "cell", "cosine4", torch.float32, 1, 5000, {}),
        ("cc3_f32_c2", 3, (24, 20, 16), "cell", "peskin4", torch.float32, 2, 5000, {}),
        ("small3_f32", 3, (9, 7, 11), "mac", "peskin4", torch.float32, None, 700, {}),
        ("mac2_f32", 2, (64, 48), "mac", "peskin4", torch.float32, None, 3000, {"seam": True}),
        ("mac2_f64", 2, (40, 33), "mac", "cosine4", torch.float64, None, 900, {}),
        ("cluster3_f32", 3, (64, 64, 64), "mac", "peskin4", torch.float32, None, 4000, {"lo": 0.4, "hi": 0.45}),
        ("roma3_f32", 3, (32, 32, 32), "mac", "roma3", torch.float32, None, 8000, {"seam": True}),
        ("bspline6_f32", 3, (32, 24, 16), "mac", "bspline6", torch.float32, None, 8000, {}),
        ("roma3_2d_f64", 2, (30, 20), "mac", "roma3", torch.float64, None, 700, {}),
        ("bspline6_cc_f32", 3, (20, 20, 20), "cell", "bspline6", torch.float32, 1, 3000, {}),
    ]
    for i, (name, dim, n, grid, kernel, dt, nc, npts, ex) in enumerate(specs):
        L = (1.0,) * dim
        comp = dt == torch.float32 and kernel in ("peskin4", "cosine4")
        p = Plan(dim, n[:dim], L, grid=grid, kernel=kernel, dtype=dt, ncomp=nc, max_points=npts, compensated=comp)
        X = _pts(10 + i, npts, dim, dt, ex.get("lo", 0.0), ex.get("hi", 1.0), ex.get("seam", False))
        g = torch.Generator().manual_seed(20 + i)
        G = torch.randn((npts, p.ncomp), generator=g, dtype=torch.float64).to(dt).cuda()
        u = torch.randn(p.grid_shape(), generator=g, dtype=torch.float64).to(dt).cuda()
        f = p.spread(X, G)
        f2 = p.spread(X, G, f=f.clone(), accumulate=True, reuse_bins=True)
        U = p.interpolate(X, u, reuse_bins=True)
        res = [f, f2, U]
        if comp:
            res.append(p.spread(X, G, compensated=True, reuse_bins=True))
        if p.ncomp == dim:
            res.append(p.pos_grad(X, u, G, reuse_bins=True))
        p.check()
        out[name] = _h(*res)
        p.close()
    # walls in z (bounded), 4-point and 6-point kernels
    for name, kernel in (("walls_peskin4", "peskin4"), ("walls_bspline6", "bspline6")):
        n = (24, 20, 16)
        p = Plan(3, n, (1.0, 1.0, 1.0), kernel=kernel, max_points=4000, bounded=(False, False, True))
        X = _pts(41, 4000, 3, torch.float32)
        g = torch.Generator().manual_seed(42)
        G = torch.randn((4000, 3), generator=g, dtype=torch.float64).float().cuda()
        u = torch.randn(p.grid_shape(), generator=g, dtype=torch.float64).float().cuda()
        f = p.spread(X, G)
        U = p.interpolate(X, u, reuse_bins=True)
        D = p.pos_grad(X, u, G, reuse_bins=True)
        p.check()
        out[name] = _h(f, U, D)
        p.close()
    # one batched wave of uneven jobs
    b = Batch(dim=3, max_jobs=4, max_points=1 << 14, max_cells=1 << 16)
    jobs, keep = [], []
    for k, (N, m) in enumerate(((8, 300), (17, 2000), (32, 5000))):
        X = _pts(50 + k, m, 3, torch.float32)
        G = torch.randn((m, 3), generator=torch.Generator().manual_seed(60 + k), dtype=torch.float64).float().cuda()
        f = torch.empty((3, N, N, N), device="cuda")
        U = torch.empty_like(X)
        keep.append((X, G, f, U))
        jobs.append(b.job_struct((N,) * 3, (1.0,) * 3, X, G=G, f=f, u=f, U=U))
    b.run(jobs)
    b.check()
    out["batch"] = _h(*[t for kk in keep for t in kk[2:]])
    b.close()
    # the interpolation that allocates nothing (its scratch is the library's fixed array);
    # it reads no error word back, so only the bit comparison with the release build speaks for it
    import ctypes
    lib = _abi.load()
    d = _abi.ib_plan_desc()
    d.dim, d.grid, d.kernel, d.dtype, d.ncomp, d.max_points, d.flags = 3, _abi.IB_GRID_MAC, 0, _abi.IB_F32, 3, 0, 0
    for k, (nn, LL) in enumerate(zip((40, 24, 17), (1.0, 0.6, 0.425))):
        d.n[k], d.L[k] = nn, LL
    X = _pts(70, 6000, 3, torch.float32, seam=True) * torch.tensor([1.0, 0.6, 0.425], device="cuda")
    u = torch.randn((3, 17, 24, 40), generator=torch.Generator().manual_seed(71), dtype=torch.float64).float().cuda()
    U = torch.empty((6000, 3), device="cuda")
    _abi.check(lib.ib_interpolate_noalloc(ctypes.byref(d), 6000, X.data_ptr(), u.data_ptr(), U.data_ptr(),
                                          torch.cuda.current_stream().cuda_stream), "ib_interpolate_noalloc")
    out["noalloc"] = _h(U)
    return out


if __name__ == "__main__":
    print(json.dumps(run_cases()))
    sys.stdout.flush()
