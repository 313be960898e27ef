"""FP64 oracle for spreading and interpolation (arXiv 2012.06646).

TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
cpu_baseline / reference leg of bench.py may import this package.  It loads
oracle/_build/liboracle.so, compiled from ib_oracle.c by build(), and wraps
each C function for numpy arrays.  It shares no code with the CUDA library
in paper_2012_06646_gb300/ and never imports it.

Every wrapped function evaluates the paper's definition directly in FP64:
  spread   -- Eq. disc-spread (serial structure of Algorithm 2)
  interp   -- Eq. disc-interp (per-point structure of Algorithm 3)
  bin_stable / cell_keys -- key computation and stable key sort of Algorithm 4 / Fig. 2
  pos_grad -- derivative of the interpolation weights with respect to X
Inputs are float64 arrays holding exactly the values the GPU path consumes
(FP32 inputs are widened, not regenerated).
"""

from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (FP64, no FMA contraction)."""
    src = os.path.join(_HERE, "ib_oracle.c")
    if not force and os.path.exists(_SO) and os.path.getmtime(_SO) >= max(
            os.path.getmtime(src), os.path.getmtime(os.path.join(_HERE, "ib_oracle.h"))):
        return _SO
    os.makedirs(_BUILD, exist_ok=True)
    tmp = _SO + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-D_DEFAULT_SOURCE", "-ffp-contract=off", "-fPIC",
                           "-shared", "-o", tmp, src, "-lm"])
    os.replace(tmp, _SO)
    return _SO


class _Grid(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("n", ctypes.c_int * 3), ("L", ctypes.c_double * 3),
                ("grid", ctypes.c_int), ("kernel", ctypes.c_int), ("ncomp", ctypes.c_int), ("bounded", ctypes.c_int)]


@dataclass(frozen=True)
class Grid:
    """Grid description: dim, points per dimension n, box sides L, grid kind, kernel, ncomp."""
    dim: int
    n: tuple
    L: tuple
    mac: bool = True
    kernel: int = 0          # 0 = standard 4-point, 1 = cosine, 2 = 3-point, 3 = 6-point B-spline
    ncomp: int | None = None
    bounded: tuple = ()      # per dimension: True for a non-periodic dimension

    @property
    def comps(self) -> int:
        return self.ncomp if self.ncomp is not None else self.dim

    @property
    def ncell(self) -> int:
        return int(np.prod(self.n[: self.dim]))

    def shape(self):
        """Component-major grid array shape [a][z][y][x] (x fastest)."""
        return (self.comps,) + tuple(reversed(self.n[: self.dim]))

    def c(self) -> _Grid:
        g = _Grid()
        g.dim = self.dim
        for b in range(3):
            g.n[b] = int(self.n[b]) if b < len(self.n) else 1
            g.L[b] = float(self.L[b]) if b < len(self.L) else 1.0
        g.grid = 1 if self.mac else 0
        g.kernel = int(self.kernel)
        g.ncomp = int(self.comps)
        g.bounded = sum(1 << b for b, v in enumerate(self.bounded) if v)
        return g


_lib = None


def lib():
    global _lib
    if _lib is None:
        path = build()
        L = ctypes.CDLL(path)
        dp = ctypes.POINTER(ctypes.c_double)
        L.or_phi.restype = ctypes.c_double
        L.or_phi.argtypes = [ctypes.c_int, ctypes.c_double]
        L.or_dphi.restype = ctypes.c_double
        L.or_dphi.argtypes = [ctypes.c_int, ctypes.c_double]
        L.or_width.restype = ctypes.c_int
        L.or_width.argtypes = [ctypes.c_int]
        L.or_cell.argtypes = [ctypes.c_double, ctypes.c_double, ctypes.c_double,
                              ctypes.POINTER(ctypes.c_longlong), dp]
        L.or_cell_keys.argtypes = [ctypes.POINTER(_Grid), ctypes.c_longlong, dp, ctypes.POINTER(ctypes.c_ulonglong)]
        L.or_bin_stable.restype = ctypes.c_longlong
        L.or_bin_stable.argtypes = [ctypes.c_longlong, ctypes.POINTER(ctypes.c_ulonglong), ctypes.c_ulonglong,
                                    ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(ctypes.c_longlong)]
        L.or_spread.argtypes = [ctypes.POINTER(_Grid), ctypes.c_longlong, dp, dp, dp, dp]
        L.or_interp.argtypes = [ctypes.POINTER(_Grid), ctypes.c_longlong, dp, dp, dp, dp]
        L.or_pos_grad.argtypes = [ctypes.POINTER(_Grid), ctypes.c_longlong, dp, dp, dp, dp, dp]
        L.or_set_mutation.argtypes = [ctypes.c_int]
        _lib = L
    return _lib


def _dp(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def phi(kernel: int, r) -> np.ndarray:
    r = np.atleast_1d(np.asarray(r, dtype=np.float64))
    return np.array([lib().or_phi(kernel, float(x)) for x in r.ravel()]).reshape(r.shape)


def width(kernel: int) -> int:
    """Support width s of the kernel (Section 3.1)."""
    return int(lib().or_width(int(kernel)))


def dphi(kernel: int, r) -> np.ndarray:
    r = np.atleast_1d(np.asarray(r, dtype=np.float64))
    return np.array([lib().or_dphi(kernel, float(x)) for x in r.ravel()]).reshape(r.shape)


def cell(X: float, scale: float, xi: float):
    i = ctypes.c_longlong()
    r = ctypes.c_double()
    lib().or_cell(float(X), float(scale), float(xi), ctypes.byref(i), ctypes.byref(r))
    return int(i.value), float(r.value)


def cell_keys(g: Grid, X) -> np.ndarray:
    X = _f64(X).reshape(-1, g.dim)
    key = np.zeros(len(X), dtype=np.uint64)
    gc = g.c()
    rc = lib().or_cell_keys(ctypes.byref(gc), len(X), _dp(X), key.ctypes.data_as(ctypes.POINTER(ctypes.c_ulonglong)))
    if rc:
        raise ValueError("invalid grid")
    return key


def bin_stable(key, nkeys: int):
    """Stable sort of point indices by key: returns (perm, start, q)."""
    key = np.ascontiguousarray(np.asarray(key, dtype=np.uint64))
    perm = np.zeros(len(key), dtype=np.int64)
    start = np.zeros(int(nkeys) + 1, dtype=np.int64)
    q = lib().or_bin_stable(len(key), key.ctypes.data_as(ctypes.POINTER(ctypes.c_ulonglong)), int(nkeys),
                            perm.ctypes.data_as(ctypes.POINTER(ctypes.c_longlong)),
                            start.ctypes.data_as(ctypes.POINTER(ctypes.c_longlong)))
    return perm, start, int(q)


def spread(g: Grid, X, G):
    """f = S G with h^-d (Eq. disc-spread); returns (f, fabs) shaped g.shape()."""
    X = _f64(X).reshape(-1, g.dim)
    G = _f64(G).reshape(len(X), g.comps)
    f = np.zeros(g.comps * g.ncell)
    fa = np.zeros_like(f)
    gc = g.c()
    if lib().or_spread(ctypes.byref(gc), len(X), _dp(X), _dp(G), _dp(f), _dp(fa)):
        raise ValueError("invalid grid")
    return f.reshape(g.shape()), fa.reshape(g.shape())


def interp(g: Grid, X, u):
    """U = S* u (Eq. disc-interp); returns (U, Uabs) shaped (n, ncomp)."""
    X = _f64(X).reshape(-1, g.dim)
    u = _f64(u).reshape(-1)
    if u.size != g.comps * g.ncell:
        raise ValueError("grid field has the wrong size")
    U = np.zeros((len(X), g.comps))
    Ua = np.zeros_like(U)
    gc = g.c()
    if lib().or_interp(ctypes.byref(gc), len(X), _dp(X), _dp(u), _dp(U), _dp(Ua)):
        raise ValueError("invalid grid")
    return U, Ua


def pos_grad(g: Grid, X, field, v):
    """D_{j,b} = sum_a v_{j,a} sum_k d/dX_b[weight] field_a[k]; returns (D, Dabs) shaped (n, dim)."""
    X = _f64(X).reshape(-1, g.dim)
    field = _f64(field).reshape(-1)
    v = _f64(v).reshape(len(X), g.comps)
    D = np.zeros((len(X), g.dim))
    Da = np.zeros_like(D)
    gc = g.c()
    if lib().or_pos_grad(ctypes.byref(gc), len(X), _dp(X), _dp(field), _dp(v), _dp(D), _dp(Da)):
        raise ValueError("invalid grid")
    return D, Da


def set_mutation(m: int) -> None:
    lib().or_set_mutation(int(m))


def inv_cell_volume(g: Grid) -> float:
    return float(np.prod([g.n[b] / g.L[b] for b in range(g.dim)]))
