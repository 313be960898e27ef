"""Tensor-level wrappers of the C ABI: argument marshalling only.

`Plan` owns an `ib_plan` (one grid description plus its device scratch) and
passes torch CUDA tensors to the C entry points as raw device pointers on
the current torch stream.  Every computation happens in the CUDA kernels of
libibgb.so; this module only checks shapes, dtypes and devices, allocates
outputs, and turns status codes into exceptions.
"""

from __future__ import annotations

import ctypes

import torch

from . import _abi
from ._abi import check

_DTYPES = {torch.float32: _abi.IB_F32, torch.float64: _abi.IB_F64}


def _stream_ptr(stream=None) -> ctypes.c_void_p:
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _ptr(t) -> ctypes.c_void_p:
    return ctypes.c_void_p(0 if t is None else t.data_ptr())


# The ib_set_allocator pair in force: (alloc, free) ctypes callbacks, or None
# for cudaMalloc / cudaFree.  Plans and batches keep a reference to the pair
# they were created with, since they free their arena through it.
_allocator = None


def set_allocator(alloc=None, free=None) -> None:
    """Arena allocator of the plans and batches created from now on (ib_set_allocator).

    alloc(nbytes) -> int device pointer (0 when out of memory, 256-byte aligned);
    free(ptr) -> None.  set_allocator() restores cudaMalloc / cudaFree.  An
    exception raised by alloc counts as out of memory.
    """
    global _allocator
    lib = _abi.load()
    if (alloc is None) != (free is None):
        raise ValueError("set_allocator needs both alloc and free, or neither")
    if alloc is None:
        check(lib.ib_set_allocator(_abi.ib_alloc_fn(), _abi.ib_free_fn(), None), "ib_set_allocator")
        _allocator = None
        return

    def _alloc(nbytes, _ctx):
        try:
            return int(alloc(int(nbytes)) or 0)
        except Exception:
            return 0

    def _free(ptr, _ctx):
        free(int(ptr))

    pair = (_abi.ib_alloc_fn(_alloc), _abi.ib_free_fn(_free))
    check(lib.ib_set_allocator(pair[0], pair[1], None), "ib_set_allocator")
    _allocator = pair


def use_torch_allocator(device=None) -> None:
    """Take plan and batch arenas from PyTorch's caching allocator on `device`."""
    dev = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
    set_allocator(lambda n: torch.cuda.caching_allocator_alloc(n, dev),
                  torch.cuda.caching_allocator_delete)


class _DeviceArray:
    """Zero-copy view of library-owned device memory through __cuda_array_interface__."""

    def __init__(self, ptr: int, n: int, typestr: str):
        self.__cuda_array_interface__ = {"shape": (n,), "typestr": typestr, "data": (ptr, False), "version": 3}


class Plan:
    """A periodic grid (dim, n, L, MAC or cell-centred, kernel, dtype, ncomp) and its scratch.

    Grid fields are tensors of shape (ncomp, n2, n1, n0) in 3-D or (ncomp, n1, n0) in 2-D;
    point arrays are (npts, dim) and (npts, ncomp).  `bounded` names the non-periodic
    dimensions (e.g. (False, False, True): walls at z = 0 and z = L).
    """

    def __init__(self, dim: int, n, L, grid: str = "mac", kernel: str = "peskin4", dtype=torch.float32,
                 ncomp: int | None = None, max_points: int = 0, compensated: bool = False, device=None,
                 bounded=(False, False, False)):
        self.lib = _abi.load()
        self.dim = int(dim)
        self.n = tuple(int(v) for v in n)[: self.dim]
        self.L = tuple(float(v) for v in L)[: self.dim]
        self.mac = grid == "mac"
        self.kernel = {"peskin4": _abi.IB_KERNEL_PESKIN4, "cosine4": _abi.IB_KERNEL_COSINE4,
                       "roma3": _abi.IB_KERNEL_ROMA3, "bspline6": _abi.IB_KERNEL_BSPLINE6}[kernel]
        self.dtype = dtype
        self.ncomp = int(ncomp) if ncomp is not None else self.dim
        self.max_points = int(max_points)
        self.device = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        d = _abi.ib_plan_desc()
        d.dim = self.dim
        for b in range(3):
            d.n[b] = self.n[b] if b < self.dim else 1
            d.L[b] = self.L[b] if b < self.dim else 1.0
        d.grid = _abi.IB_GRID_MAC if self.mac else _abi.IB_GRID_CELL_CENTERED
        d.kernel = self.kernel
        d.dtype = _DTYPES[dtype]
        d.ncomp = self.ncomp
        d.max_points = self.max_points
        d.flags = _abi.IB_PLAN_COMPENSATED if compensated else 0
        for b, flag in enumerate((_abi.IB_PLAN_BOUNDED_X, _abi.IB_PLAN_BOUNDED_Y, _abi.IB_PLAN_BOUNDED_Z)):
            if b < len(bounded) and bounded[b]:
                d.flags |= flag
        self.bounded = tuple(bool(v) for v in bounded)
        self.desc = d
        h = ctypes.c_void_p()
        self._allocator = _allocator
        with torch.cuda.device(self.device):
            check(self.lib.ib_plan_create(ctypes.byref(d), ctypes.byref(h)), "ib_plan_create")
        self.handle = h
        # Incremented by every call that replaces the plan's bins (binning, a call
        # without reuse_bins, the paper's algorithms, an in-place position update):
        # callers that keep bins across calls compare it to decide whether to re-bin.
        self.bin_epoch = 0

    # -- helpers ---------------------------------------------------------
    def grid_shape(self):
        return (self.ncomp,) + tuple(reversed(self.n))

    def footprint(self) -> int:
        size = ctypes.c_size_t()
        check(self.lib.ib_plan_footprint(ctypes.byref(self.desc), ctypes.byref(size)), "ib_plan_footprint")
        return size.value

    def _points(self, X):
        if X.device != self.device or X.dtype != self.dtype or not X.is_contiguous():
            raise ValueError("X must be a contiguous tensor of the plan's dtype on the plan's device")
        if X.dim() != 2 or X.shape[1] != self.dim:
            raise ValueError(f"X must have shape (npts, {self.dim})")
        return X.shape[0]

    def _check(self, t, shape, name):
        if t.device != self.device or t.dtype != self.dtype or not t.is_contiguous():
            raise ValueError(f"{name} must be a contiguous tensor of the plan's dtype on the plan's device")
        if tuple(t.shape) != tuple(shape):
            raise ValueError(f"{name} must have shape {tuple(shape)}, got {tuple(t.shape)}")

    def _new(self, shape):
        return torch.empty(shape, dtype=self.dtype, device=self.device)

    # -- entry points ------------------------------------------------------
    def bin(self, X, stream=None):
        n = self._points(X)
        check(self.lib.ib_bin(self.handle, n, _ptr(X), _stream_ptr(stream)), "ib_bin")
        self.bin_epoch += 1

    def spread(self, X, G, f=None, accumulate=False, compensated=False, reuse_bins=False, adjoint=False,
               overlap_previous=False, stream=None):
        """ib_spread.  overlap_previous (IB_OVERLAP_PREVIOUS, with reuse_bins): the library call just before
        on the stream wrote nothing this one reads (X, G, the bins), so spreading may start during its tail."""
        n = self._points(X)
        self._check(G, (n, self.ncomp), "G")
        if f is None:
            f = self._new(self.grid_shape())
        self._check(f, self.grid_shape(), "f")
        flags = ((_abi.IB_ACCUMULATE if accumulate else 0) | (_abi.IB_COMPENSATED if compensated else 0)
                 | (_abi.IB_REUSE_BINS if reuse_bins else 0) | (_abi.IB_ADJOINT if adjoint else 0)
                 | (_abi.IB_OVERLAP_PREVIOUS if overlap_previous else 0))
        check(self.lib.ib_spread(self.handle, n, _ptr(X), _ptr(G), _ptr(f), flags, _stream_ptr(stream)), "ib_spread")
        if not reuse_bins:
            self.bin_epoch += 1
        return f

    def spread_paper(self, X, G, algorithm: int = 4, beta: int = 8, f=None, buffer=None, stream=None):
        """The paper's spreading algorithm 4, 5 or 6 (comparators of `spread`): f = S G.

        Algorithm 5 uses `buffer` (beta grids of the plan's dtype; allocated here if None)."""
        n = self._points(X)
        self._check(G, (n, self.ncomp), "G")
        if f is None:
            f = self._new(self.grid_shape())
        self._check(f, self.grid_shape(), "f")
        if algorithm == 5 and buffer is None:
            buffer = torch.empty((beta,) + tuple(reversed(self.n)), dtype=self.dtype, device=self.device)
        self.bin_epoch += 1
        check(self.lib.ib_spread_paper(self.handle, n, _ptr(X), _ptr(G), _ptr(f), int(algorithm), int(beta),
                                       _ptr(buffer), _stream_ptr(stream)), "ib_spread_paper")
        return f

    def interpolate(self, X, u, U=None, reuse_bins=False, adjoint=False, stream=None):
        n = self._points(X)
        self._check(u, self.grid_shape(), "u")
        if U is None:
            U = self._new((n, self.ncomp))
        self._check(U, (n, self.ncomp), "U")
        flags = (_abi.IB_REUSE_BINS if reuse_bins else 0) | (_abi.IB_ADJOINT if adjoint else 0)
        if not reuse_bins:
            self.bin_epoch += 1
        check(self.lib.ib_interpolate(self.handle, n, _ptr(X), _ptr(u), _ptr(U), flags, _stream_ptr(stream)),
              "ib_interpolate")
        return U

    def pos_grad(self, X, field, v, scale: float = 1.0, D=None, reuse_bins=False, spread=False, stream=None):
        """ib_pos_grad; spread=True differentiates spreading's weights (IB_SPREAD_GRAD:
        the library multiplies scale by h^-d)."""
        n = self._points(X)
        self._check(field, self.grid_shape(), "field")
        self._check(v, (n, self.ncomp), "v")
        if D is None:
            D = self._new((n, self.dim))
        self._check(D, (n, self.dim), "D")
        flags = (_abi.IB_REUSE_BINS if reuse_bins else 0) | (_abi.IB_SPREAD_GRAD if spread else 0)
        if not reuse_bins:
            self.bin_epoch += 1
        check(self.lib.ib_pos_grad(self.handle, n, _ptr(X), _ptr(field), _ptr(v), float(scale), _ptr(D), flags,
                                   _stream_ptr(stream)), "ib_pos_grad")
        return D

    def advect(self, X, U, dt: float, out=None, overlap_previous=False, stream=None):
        """ib_advect: out = X + dt U, wrapped.  overlap_previous (IB_OVERLAP_PREVIOUS): the library call just
        before on the stream wrote neither X nor U (e.g. a spread), so the update may start during its tail."""
        n = self._points(X)
        self._check(U, (n, self.dim), "U")
        if out is None:
            out = self._new((n, self.dim))
        self._check(out, (n, self.dim), "out")
        if out.data_ptr() == X.data_ptr():
            self.bin_epoch += 1
        flags = _abi.IB_OVERLAP_PREVIOUS if overlap_previous else 0
        check(self.lib.ib_advect(self.handle, n, _ptr(X), _ptr(U), float(dt), _ptr(out), flags,
                                 _stream_ptr(stream)), "ib_advect")
        return out

    def check(self, stream=None) -> None:
        """Synchronise and raise if a kernel flagged a non-finite or out-of-range position."""
        check(self.lib.ib_plan_check(self.handle, _stream_ptr(stream)), "ib_plan_check")

    def bins(self):
        """(perm, cell_start) of the last binning, as int64 copies (perm: npts, cell_start: ncell + 2)."""
        perm = ctypes.c_void_p()
        start = ctypes.c_void_p()
        ncell = ctypes.c_longlong()
        npts = ctypes.c_longlong()
        check(self.lib.ib_plan_bins(self.handle, ctypes.byref(perm), ctypes.byref(start), ctypes.byref(ncell),
                                    ctypes.byref(npts)), "ib_plan_bins")
        if npts.value < 0:
            raise RuntimeError("no binning has run on this plan")
        torch.cuda.current_stream().synchronize()
        p = torch.as_tensor(_DeviceArray(perm.value, npts.value, "<i4"), device=self.device)
        s = torch.as_tensor(_DeviceArray(start.value, ncell.value + 2, "<i4"), device=self.device)
        return p.to(torch.int64), s.to(torch.int64)

    def close(self):
        if getattr(self, "handle", None):
            self.lib.ib_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Stokes:
    """An `ib_stokes`: the periodic MAC-grid Stokes solve of the IB step (e).

    `solve(f, u_old, rho_over_k, mu)` returns u with (rho/k) u + G p - mu L u = (rho/k) u_old + f
    and D u = 0; fields have the Plan grid shape (dim, n2, n1, n0) / (dim, n1, n0).
    """

    def __init__(self, dim: int, n, L, dtype=torch.float32, device=None):
        self.lib = _abi.load()
        self.dim = int(dim)
        self.n = tuple(int(v) for v in n)[: self.dim]
        self.L = tuple(float(v) for v in L)[: self.dim]
        self.dtype = dtype
        self.device = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        d = _abi.ib_plan_desc()
        d.dim = self.dim
        for b in range(3):
            d.n[b] = self.n[b] if b < self.dim else 1
            d.L[b] = self.L[b] if b < self.dim else 1.0
        d.grid = _abi.IB_GRID_MAC
        d.kernel = _abi.IB_KERNEL_PESKIN4
        d.dtype = _DTYPES[dtype]
        d.ncomp = self.dim
        self.desc = d
        h = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            check(self.lib.ib_stokes_create(ctypes.byref(d), ctypes.byref(h)), "ib_stokes_create")
        self.handle = h

    def grid_shape(self):
        return (self.dim,) + tuple(reversed(self.n))

    def _check(self, t, name):
        if t.device != self.device or t.dtype != self.dtype or not t.is_contiguous():
            raise ValueError(f"{name} must be a contiguous tensor of the solver's dtype on its device")
        if tuple(t.shape) != self.grid_shape():
            raise ValueError(f"{name} must have shape {self.grid_shape()}, got {tuple(t.shape)}")

    def solve(self, f, u_old=None, rho_over_k: float = 1.0, mu: float = 1.0, u=None, stream=None):
        self._check(f, "f")
        if u_old is not None:
            self._check(u_old, "u_old")
        if u is None:
            u = torch.empty(self.grid_shape(), dtype=self.dtype, device=self.device)
        self._check(u, "u")
        check(self.lib.ib_stokes_solve(self.handle, _ptr(f), _ptr(u_old), _ptr(u), float(rho_over_k), float(mu),
                                       _stream_ptr(stream)), "ib_stokes_solve")
        return u

    def close(self):
        if getattr(self, "handle", None):
            self.lib.ib_stokes_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """An `ib_batch`: one wave of independent spread + interpolate jobs per `run` call."""

    def __init__(self, dim=3, grid="mac", kernel="peskin4", dtype=torch.float32, ncomp=None, max_jobs=64,
                 max_points=1 << 22, max_cells=1 << 24, max_tiles=None, host_io=False, device=None):
        self.lib = _abi.load()
        self.dim = dim
        self.ncomp = ncomp if ncomp is not None else dim
        self.dtype = dtype
        self.device = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        d = _abi.ib_batch_desc()
        d.dim = dim
        d.grid = _abi.IB_GRID_MAC if grid == "mac" else _abi.IB_GRID_CELL_CENTERED
        d.kernel = {"peskin4": _abi.IB_KERNEL_PESKIN4, "cosine4": _abi.IB_KERNEL_COSINE4}[kernel]
        d.dtype = _DTYPES[dtype]
        d.ncomp = self.ncomp
        d.max_jobs = int(max_jobs)
        d.max_points = int(max_points)
        d.max_cells = int(max_cells)
        d.max_tiles = int(max_tiles if max_tiles is not None else max_cells // 512 + 8 * max_jobs)
        d.flags = _abi.IB_BATCH_HOST_IO if host_io else 0
        self.desc = d
        h = ctypes.c_void_p()
        self._allocator = _allocator
        with torch.cuda.device(self.device):
            check(self.lib.ib_batch_create(ctypes.byref(d), ctypes.byref(h)), "ib_batch_create")
        self.handle = h

    def footprint(self) -> int:
        size = ctypes.c_size_t()
        check(self.lib.ib_batch_footprint(ctypes.byref(self.desc), ctypes.byref(size)), "ib_batch_footprint")
        return size.value

    def job_struct(self, n, L, X, G=None, f=None, u=None, U=None) -> _abi.ib_job:
        j = _abi.ib_job()
        for b in range(3):
            j.n[b] = int(n[b]) if b < self.dim else 1
            j.L[b] = float(L[b]) if b < self.dim else 1.0
        j.npts = X.shape[0]
        j.X = X.data_ptr()
        j.G = G.data_ptr() if G is not None else None
        j.f = f.data_ptr() if f is not None else None
        j.u = u.data_ptr() if u is not None else None
        j.U = U.data_ptr() if U is not None else None
        return j

    def job_footprint(self, job: _abi.ib_job):
        size = ctypes.c_size_t()
        tiles = ctypes.c_longlong()
        check(self.lib.ib_batch_job_footprint(ctypes.byref(self.desc), ctypes.byref(job), ctypes.byref(size),
                                              ctypes.byref(tiles)), "ib_batch_job_footprint")
        return size.value, tiles.value

    def run(self, jobs, stream=None) -> None:
        arr = (_abi.ib_job * len(jobs))(*jobs)
        check(self.lib.ib_batch_run(self.handle, len(jobs), arr, 0, _stream_ptr(stream)), "ib_batch_run")

    def run_host(self, jobs, stream=None) -> None:
        """One served wave with host-resident data: jobs = [(n, L, X, G, U)], X/G/U host tensors
        (pinned for asynchronous copies) of shapes (npts, dim), (npts, ncomp), (npts, ncomp)."""
        arr = (_abi.ib_host_job * len(jobs))()
        for j, (n, L, X, G, U) in zip(arr, jobs):
            for b in range(3):
                j.n[b] = int(n[b]) if b < self.dim else 1
                j.L[b] = float(L[b]) if b < self.dim else 1.0
            j.npts = X.shape[0]
            j.X = X.data_ptr()
            j.G = G.data_ptr()
            j.U = U.data_ptr()
        check(self.lib.ib_batch_run_host(self.handle, len(jobs), arr, _stream_ptr(stream)), "ib_batch_run_host")

    def check(self, stream=None) -> None:
        check(self.lib.ib_batch_check(self.handle, _stream_ptr(stream)), "ib_batch_check")

    def status(self, stream=None) -> int:
        """ib_batch_check without raising: the status code of the error word (read and cleared)."""
        return int(self.lib.ib_batch_check(self.handle, _stream_ptr(stream)))

    def wave_status(self) -> int:
        """ib_batch_wave_status: the error word as the last run_host wave left it (no synchronisation;
        valid once that wave's stream has passed it)."""
        return int(self.lib.ib_batch_wave_status(self.handle))

    def close(self):
        if getattr(self, "handle", None):
            self.lib.ib_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
