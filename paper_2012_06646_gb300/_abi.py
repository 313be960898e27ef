"""ctypes declarations of the C ABI in include/ib.h, under the same names.

Loads paper_2012_06646_gb300/_lib/libibgb.so (built by build.py).  There is
no fallback: if the library is missing, loading raises, because every step
of the path runs in the CUDA kernels of that library.
"""

from __future__ import annotations

import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libibgb.so")
# The index-checking build (build(debug_bounds=True)); loaded instead of the
# release library when the environment sets IBGB_DEBUG_BOUNDS=1.
DEBUG_LIB_PATH = os.path.join(_HERE, "_lib_debug", "libibgb.so")


def default_path() -> str:
    return DEBUG_LIB_PATH if os.environ.get("IBGB_DEBUG_BOUNDS") == "1" else LIB_PATH

IB_OK = 0
IB_ERR_INVALID_ARG = 1
IB_ERR_OOM = 2
IB_ERR_CUDA = 3
IB_ERR_TIMEOUT = 4
IB_ERR_CAPACITY = 5
IB_ERR_NOT_IMPLEMENTED = 6
IB_ERR_NONFINITE = 7
IB_ERR_RANGE = 8
IB_ERR_NO_BINS = 9
IB_ERR_BINS_STALE = 10
IB_ERR_BOUNDS = 11

IB_KERNEL_PESKIN4 = 0
IB_KERNEL_COSINE4 = 1
IB_KERNEL_ROMA3 = 2
IB_KERNEL_BSPLINE6 = 3
IB_GRID_CELL_CENTERED = 0
IB_GRID_MAC = 1
IB_F32 = 0
IB_F64 = 1

IB_PLAN_COMPENSATED = 0x1
IB_PLAN_BOUNDED_X = 0x2
IB_PLAN_BOUNDED_Y = 0x4
IB_PLAN_BOUNDED_Z = 0x8
IB_ACCUMULATE = 0x1
IB_COMPENSATED = 0x2
IB_REUSE_BINS = 0x4
IB_ADJOINT = 0x8
IB_SPREAD_GRAD = 0x10
IB_OVERLAP_PREVIOUS = 0x20

IB_BATCH_HOST_IO = 0x1

IB_PAPER_ALG4 = 4
IB_PAPER_ALG5 = 5
IB_PAPER_ALG6 = 6

IB_NOALLOC_MAX_CELLS = 1 << 21
IB_NOALLOC_MAX_POINTS = 1 << 20


class ib_plan_desc(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("n", ctypes.c_int * 3), ("L", ctypes.c_double * 3),
                ("grid", ctypes.c_int), ("kernel", ctypes.c_int), ("dtype", ctypes.c_int),
                ("ncomp", ctypes.c_int), ("max_points", ctypes.c_longlong), ("flags", ctypes.c_uint)]


class ib_batch_desc(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("grid", ctypes.c_int), ("kernel", ctypes.c_int),
                ("dtype", ctypes.c_int), ("ncomp", ctypes.c_int), ("max_jobs", ctypes.c_int),
                ("max_points", ctypes.c_longlong), ("max_cells", ctypes.c_longlong),
                ("max_tiles", ctypes.c_longlong), ("flags", ctypes.c_uint)]


class ib_job(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int * 3), ("L", ctypes.c_double * 3), ("npts", ctypes.c_longlong),
                ("X", ctypes.c_void_p), ("G", ctypes.c_void_p), ("f", ctypes.c_void_p),
                ("u", ctypes.c_void_p), ("U", ctypes.c_void_p)]


class ib_host_job(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int * 3), ("L", ctypes.c_double * 3), ("npts", ctypes.c_longlong),
                ("X", ctypes.c_void_p), ("G", ctypes.c_void_p), ("U", ctypes.c_void_p)]


_vp = ctypes.c_void_p
_ll = ctypes.c_longlong
_st = ctypes.c_int

# ib_alloc_fn / ib_free_fn of ib_set_allocator (called with no argument: NULL)
ib_alloc_fn = ctypes.CFUNCTYPE(_vp, ctypes.c_size_t, _vp)
ib_free_fn = ctypes.CFUNCTYPE(None, _vp, _vp)

# name -> (restype, argtypes)
SIGNATURES = {
    "ib_plan_footprint": (_st, [ctypes.POINTER(ib_plan_desc), ctypes.POINTER(ctypes.c_size_t)]),
    "ib_plan_create": (_st, [ctypes.POINTER(ib_plan_desc), ctypes.POINTER(_vp)]),
    "ib_plan_destroy": (_st, [_vp]),
    "ib_bin": (_st, [_vp, _ll, _vp, _vp]),
    "ib_spread": (_st, [_vp, _ll, _vp, _vp, _vp, ctypes.c_uint, _vp]),
    "ib_interpolate": (_st, [_vp, _ll, _vp, _vp, _vp, ctypes.c_uint, _vp]),
    "ib_pos_grad": (_st, [_vp, _ll, _vp, _vp, _vp, ctypes.c_double, _vp, ctypes.c_uint, _vp]),
    "ib_advect": (_st, [_vp, _ll, _vp, _vp, ctypes.c_double, _vp, ctypes.c_uint, _vp]),
    "ib_plan_check": (_st, [_vp, _vp]),
    "ib_plan_bins": (_st, [_vp, ctypes.POINTER(_vp), ctypes.POINTER(_vp), ctypes.POINTER(_ll), ctypes.POINTER(_ll)]),
    "ib_spread_paper": (_st, [_vp, _ll, _vp, _vp, _vp, ctypes.c_int, ctypes.c_int, _vp, _vp]),
    "ib_batch_footprint": (_st, [ctypes.POINTER(ib_batch_desc), ctypes.POINTER(ctypes.c_size_t)]),
    "ib_batch_job_footprint": (_st, [ctypes.POINTER(ib_batch_desc), ctypes.POINTER(ib_job),
                                     ctypes.POINTER(ctypes.c_size_t), ctypes.POINTER(_ll)]),
    "ib_batch_create": (_st, [ctypes.POINTER(ib_batch_desc), ctypes.POINTER(_vp)]),
    "ib_batch_destroy": (_st, [_vp]),
    "ib_batch_run": (_st, [_vp, ctypes.c_int, ctypes.POINTER(ib_job), ctypes.c_uint, _vp]),
    "ib_slab_halo_bytes": (_st, [_vp, ctypes.c_uint, ctypes.POINTER(ctypes.c_size_t)]),
    "ib_slab_owner": (_st, [_vp, _ll, _vp, ctypes.c_int, ctypes.POINTER(ctypes.c_int), _vp, _vp]),
    "ib_slab_spread": (_st, [_vp, _ll, _vp, _vp, ctypes.c_int, ctypes.c_int, _vp, _vp, ctypes.c_uint, _vp]),
    "ib_slab_combine": (_st, [_vp, _vp, ctypes.c_int, ctypes.c_int, _vp, _vp, ctypes.c_uint, _vp]),
    "ib_batch_check": (_st, [_vp, _vp]),
    "ib_batch_wave_status": (_st, [_vp]),
    "ib_batch_run_host": (_st, [_vp, ctypes.c_int, ctypes.POINTER(ib_host_job), _vp]),
    "ib_interpolate_noalloc": (_st, [ctypes.POINTER(ib_plan_desc), _ll, _vp, _vp, _vp, _vp]),
    "ib_stokes_create": (_st, [ctypes.POINTER(ib_plan_desc), ctypes.POINTER(_vp)]),
    "ib_stokes_solve": (_st, [_vp, _vp, _vp, _vp, ctypes.c_double, ctypes.c_double, _vp]),
    "ib_stokes_destroy": (_st, [_vp]),
    "ib_set_allocator": (_st, [ib_alloc_fn, ib_free_fn, _vp]),
    "ib_selftest_bounded_wait": (_st, [_vp]),
    "ib_status_string": (ctypes.c_char_p, [_st]),
    "ib_version": (ctypes.c_char_p, []),
}

_lib = None


def load(path: str | None = None):
    """Load libibgb.so and declare every entry point; raises if the library is missing."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or default_path()
    if not os.path.exists(path):
        raise RuntimeError(f"CUDA library {path} is missing: build it with paper_2012_06646_gb300.build.build() "
                           "(there is no CPU fallback)")
    lib = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


class IBError(RuntimeError):
    def __init__(self, status: int, where: str = ""):
        self.status = int(status)
        name = load().ib_status_string(self.status).decode()
        super().__init__(f"{where}: {name}" if where else name)


def check(status: int, where: str = "") -> None:
    if status != IB_OK:
        raise IBError(status, where)
