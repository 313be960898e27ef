"""The periodic MAC-grid Stokes solve of the IB step (e) through the C ABI
(ib_stokes_create / ib_stokes_solve), against the FP64 oracle
oracle/stokes.py on the same seeded inputs, element by element.

Tolerances.  FP64: 1e-11 max|u_ref| (the transforms' rounding, about
eps log2(N) of the field's scale, far below).  FP32: 1e-5 max|u_ref|.  A
cuFFT transform of N points carries a relative error of order eps log2(N)
(eps = 6e-8, log2(N) <= 21 at 128^3, so about 1.3e-6 of the field's norm);
the per-mode arithmetic adds a few eps; the worst element is a few times the
rms error, which stays under 1e-5 of the largest value.  The discrete
divergence of the FP32 result is bounded by the same relative error times
max|u| / h.
"""
import ctypes

import numpy as np
import pytest
import torch

import ib_inputs
from _gpu import dev, host
from oracle import stokes

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def S():
    from paper_2012_06646_gb300 import build
    build()
    from paper_2012_06646_gb300.plan import Stokes
    return Stokes


CASES = [
    # n, L, rho/k, mu, with u_old, dtype
    ((17, 20, 24), (1.0, 1.2, 1.4), 2.0, 0.05, True, np.float64),
    ((32, 24, 40), (1.0, 0.75, 1.25), 1.0, 0.01, True, np.float32),
    ((33, 16), (1.0, 0.5), 0.0, 1.0, False, np.float64),
    ((64, 40), (2.0, 1.25), 4.0, 0.1, True, np.float32),
    ((2, 2, 2), (1.0, 1.0, 1.0), 1.0, 1.0, True, np.float64),
    ((128, 128, 128), (1.0, 1.0, 1.0), 1.0e3, 1.0e-2, True, np.float32),
    # n2 a power of two: (y, x) plane transforms and the z-column kernel
    ((24, 20, 16), (1.0, 0.8, 0.5), 3.0, 0.2, True, np.float64),
    ((17, 12, 32), (1.0, 1.0, 2.0), 1.0, 0.05, True, np.float32),      # odd n0: a partial block of kx
    ((8, 6, 256), (0.25, 0.2, 1.0), 0.0, 1.0, False, np.float32),     # the largest n2 of that path, steady
    ((40, 33, 4), (1.0, 1.0, 0.1), 10.0, 0.01, True, np.float64),
]


def _ids(c):
    return f"{len(c[0])}d-{'x'.join(map(str, c[0]))}-a{c[2]}-{np.dtype(c[5]).name}"


@pytest.mark.parametrize("case", CASES, ids=[_ids(c) for c in CASES])
def test_stokes_matches_oracle(S, case):
    n, L, alpha, mu, with_old, dtype = case
    dim = len(n)
    shape = (dim,) + tuple(reversed(n))
    f = ib_inputs.normal_array(sum(n), shape, dtype=dtype, purpose="f")
    u_old = ib_inputs.normal_array(sum(n) + 1, shape, dtype=dtype, purpose="u") if with_old else None
    want = stokes.solve(f.astype(np.float64), n, L, alpha, mu,
                        None if u_old is None else u_old.astype(np.float64))
    solver = S(dim, n, L, dtype=torch.float64 if dtype == np.float64 else torch.float32)
    got = host(solver.solve(dev(f), None if u_old is None else dev(u_old), alpha, mu)).astype(np.float64)
    scale = np.max(np.abs(want))
    rel = 1e-11 if dtype == np.float64 else 1e-5
    err = np.abs(got - want)
    assert err.max() <= rel * scale, f"max err {err.max():.3e} vs {rel * scale:.3e}"
    h = min(L[b] / n[b] for b in range(dim))
    assert np.max(np.abs(stokes.div(got, n, L))) <= 4 * rel * scale / h
    solver.close()


@pytest.mark.parametrize("n", [(20, 16, 12), (20, 16, 16)])
def test_stokes_in_place_and_repeated(S, n):
    """u may alias u_old; repeated solves on one object give identical results (both solve paths)."""
    L = (1.0, 0.8, 0.6)
    shape = (3,) + tuple(reversed(n))
    f = dev(ib_inputs.normal_array(5, shape, purpose="f"))
    u0 = dev(ib_inputs.normal_array(6, shape, purpose="u"))
    solver = S(3, n, L)
    a = solver.solve(f, u0, 3.0, 0.2)
    b = solver.solve(f, u0, 3.0, 0.2)
    u = u0.clone()
    solver.solve(f, u, 3.0, 0.2, u=u)
    torch.cuda.synchronize()
    assert torch.equal(a, b) and torch.equal(a, u)
    solver.close()


def test_stokes_argument_errors(S):
    from paper_2012_06646_gb300 import _abi
    lib = _abi.load()
    solver = S(2, (8, 8), (1.0, 1.0))
    f = torch.zeros((2, 8, 8), device="cuda")
    u = torch.empty_like(f)
    st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for rk, mu in [(0.0, 0.0), (-1.0, 1.0), (1.0, -0.5), (float("nan"), 1.0), (1.0, float("inf"))]:
        assert lib.ib_stokes_solve(solver.handle, ctypes.c_void_p(f.data_ptr()), None,
                                   ctypes.c_void_p(u.data_ptr()), rk, mu, st) == _abi.IB_ERR_INVALID_ARG
    assert lib.ib_stokes_solve(solver.handle, None, None, ctypes.c_void_p(u.data_ptr()), 1.0, 1.0, st) == \
        _abi.IB_ERR_INVALID_ARG
    solver.close()
