"""The paper's parallel spreading algorithms (Algorithm 4 and the buffered
Algorithms 5 and 6), run through the C ABI as comparators of ib_spread:
parity with the FP64 oracle, exact agreement between the variants where the
summation order is the same, and argument checks."""
import ctypes

import numpy as np
import pytest
import torch

import ib_inputs
from _gpu import FLOOR32, FLOOR64, assert_spread_close, dev, host

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    from paper_2012_06646_gb300 import build
    build()
    from paper_2012_06646_gb300.plan import Plan
    return Plan


CASES = [
    # dim, n, L, mac, kernel, ncomp, npts, dtype
    (3, (24, 20, 28), (1.0, 0.8, 1.2), True, 0, 3, 2000, np.float32),
    (3, (16, 16, 16), (1.0, 1.0, 1.0), False, 1, 1, 1500, np.float32),
    (3, (12, 12, 12), (1.0, 1.0, 1.0), True, 0, 3, 800, np.float64),
    (2, (64, 40), (1.0, 0.625), True, 0, 2, 1000, np.float32),
    (2, (64, 64), (1.0, 1.0), False, 0, 2, 1000, np.float64),
]


@pytest.mark.parametrize("case", CASES, ids=[f"{c[0]}d-{'x'.join(map(str, c[1]))}-{'mac' if c[3] else 'cc'}"
                                             f"-c{c[5]}-{np.dtype(c[7]).name}" for c in CASES])
def test_paper_algorithms_match_oracle(P, orc, case):
    dim, n, L, mac, kernel, ncomp, npts, dtype = case
    X = ib_inputs.uniform_points(sum(n), npts, L, dim, dtype=dtype)
    G = ib_inputs.normal_array(sum(n) + 1, (npts, ncomp), dtype=dtype)
    tdt = torch.float32 if dtype == np.float32 else torch.float64
    plan = P(dim, n, L, grid="mac" if mac else "cc", kernel="peskin4" if kernel == 0 else "cosine4", dtype=tdt,
             ncomp=ncomp, max_points=npts)
    g = orc.Grid(dim=dim, n=n, L=L, mac=mac, kernel=kernel, ncomp=ncomp)
    f_ref, fabs = orc.spread(g, X, G)
    rel, floor = (1e-5, FLOOR32) if dtype == np.float32 else (1e-12, FLOOR64)
    Xd, Gd = dev(X), dev(G)
    S = 4 ** dim
    f4 = host(plan.spread_paper(Xd, Gd, algorithm=4))
    assert_spread_close(f4, f_ref, fabs, rel, floor, what="algorithm 4")
    for beta in (1, 3, 8, S):
        f5 = host(plan.spread_paper(Xd, Gd, algorithm=5, beta=beta))
        assert_spread_close(f5, f_ref, fabs, rel, floor, what=f"algorithm 5, beta {beta}")
        f6 = host(plan.spread_paper(Xd, Gd, algorithm=6, beta=beta))
        assert np.array_equal(f6, f5), "algorithm 6 differs from algorithm 5 with the same beta"
        if beta == 1:   # one buffer filled shift by shift: the order of algorithm 4
            assert np.array_equal(f5, f4), "algorithm 5 with beta 1 differs from algorithm 4"
    # the tile kernels agree within the tolerance too
    f = host(plan.spread(Xd, Gd))
    assert_spread_close(f, f_ref, fabs, rel, floor)


def test_paper_algorithms_reproducible_and_checked(P):
    from paper_2012_06646_gb300 import _abi
    from paper_2012_06646_gb300._abi import IBError
    n, npts = (32, 32, 32), 20000
    plan = P(3, n, (1.0, 1.0, 1.0), max_points=npts)
    X = dev(ib_inputs.uniform_points(41, npts, (1.0, 1.0, 1.0), 3))
    G = dev(ib_inputs.normal_array(42, (npts, 3)))
    a = host(plan.spread_paper(X, G, algorithm=5, beta=8))
    b = host(plan.spread_paper(X, G, algorithm=5, beta=8))
    assert np.array_equal(a, b)
    lib = plan.lib
    f = torch.empty(plan.grid_shape(), dtype=torch.float32, device="cuda")
    s = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    call = lambda alg, beta, buf: lib.ib_spread_paper(plan.handle, npts, ctypes.c_void_p(X.data_ptr()),
                                                      ctypes.c_void_p(G.data_ptr()), ctypes.c_void_p(f.data_ptr()),
                                                      alg, beta, buf, s)
    assert call(7, 8, None) == _abi.IB_ERR_INVALID_ARG
    assert call(5, 0, ctypes.c_void_p(f.data_ptr())) == _abi.IB_ERR_INVALID_ARG
    assert call(5, 65, ctypes.c_void_p(f.data_ptr())) == _abi.IB_ERR_INVALID_ARG
    assert call(5, 8, None) == _abi.IB_ERR_INVALID_ARG
    assert call(6, 65, None) == _abi.IB_ERR_INVALID_ARG
    # the comparators re-bin by component cells: later calls cannot reuse those bins
    with pytest.raises(IBError) as e:
        plan.spread(X, G, reuse_bins=True)
    assert e.value.status == _abi.IB_ERR_NO_BINS
