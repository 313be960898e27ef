"""CPU-side checks of the boundary: the library loads without a GPU, exports every
entry point include/ib.h declares, and validates arguments on the host."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def abi():
    from paper_2012_06646_gb300.build import build
    build()
    from paper_2012_06646_gb300 import _abi
    return _abi


def header_functions():
    text = open(os.path.join(ROOT, "include", "ib.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(ib_\w+)\s*\(", text, flags=re.M)))


def test_every_declared_symbol_is_exported(abi):
    names = header_functions()
    assert len(names) >= 18
    lib = ctypes.CDLL(abi.LIB_PATH)
    for name in names:
        assert hasattr(lib, name), f"{name} declared in include/ib.h but not exported"
    assert sorted(abi.SIGNATURES) == names


def test_only_the_c_abi_is_exported(abi):
    # The linker version script keeps the internal C++ functions (and the static CUDA
    # runtime) local: the dynamic symbol table defines exactly the header's functions.
    import shutil
    import subprocess
    nm = shutil.which("nm")
    if nm is None:
        pytest.skip("nm not available")
    out = subprocess.run([nm, "-D", "--defined-only", abi.LIB_PATH], capture_output=True, text=True, check=True)
    funcs = sorted(ln.split()[-1] for ln in out.stdout.splitlines() if len(ln.split()) == 3 and ln.split()[1] == "T")
    assert funcs == header_functions()


def _desc(abi, **kw):
    d = abi.ib_plan_desc()
    d.dim = kw.get("dim", 3)
    for b, v in enumerate(kw.get("n", (128, 128, 128))):
        d.n[b] = v
    for b, v in enumerate(kw.get("L", (1.0, 1.0, 1.0))):
        d.L[b] = v
    d.grid = kw.get("grid", abi.IB_GRID_MAC)
    d.kernel = kw.get("kernel", abi.IB_KERNEL_PESKIN4)
    d.dtype = kw.get("dtype", abi.IB_F32)
    d.ncomp = kw.get("ncomp", 3)
    d.max_points = kw.get("max_points", 10 ** 6)
    d.flags = kw.get("flags", 0)
    return d


def test_footprint_and_validation_on_host(abi):
    lib = abi.load()
    size = ctypes.c_size_t()
    assert lib.ib_plan_footprint(ctypes.byref(_desc(abi)), ctypes.byref(size)) == abi.IB_OK
    # 128^3 MAC, 10^6 points: cells 8.4 MB, point arrays 20 MB, boxes 4096 x 3 x 12^3 x 4 B (84.9 MB)
    assert 105e6 < size.value < 120e6
    comp = ctypes.c_size_t()
    assert lib.ib_plan_footprint(ctypes.byref(_desc(abi, flags=abi.IB_PLAN_COMPENSATED)), ctypes.byref(comp)) == 0
    assert comp.value > size.value
    bad = [dict(dim=4), dict(ncomp=2), dict(ncomp=5, grid=abi.IB_GRID_CELL_CENTERED), dict(n=(0, 4, 4)),
           dict(L=(1.0, -1.0, 1.0)), dict(max_points=-1), dict(flags=0x80), dict(kernel=7), dict(dtype=3),
           dict(n=(2048, 2048, 1024))]
    h = ctypes.c_void_p()
    for kw in bad:
        assert lib.ib_plan_footprint(ctypes.byref(_desc(abi, **kw)), ctypes.byref(size)) == abi.IB_ERR_INVALID_ARG, kw
        assert lib.ib_plan_create(ctypes.byref(_desc(abi, **kw)), ctypes.byref(h)) == abi.IB_ERR_INVALID_ARG, kw
    assert lib.ib_spread(None, 0, None, None, None, 0, None) == abi.IB_ERR_INVALID_ARG
    assert lib.ib_batch_run(None, 0, None, 0, None) == abi.IB_ERR_INVALID_ARG
    assert lib.ib_plan_destroy(None) == abi.IB_OK
    assert lib.ib_status_string(abi.IB_ERR_NO_BINS) == b"IB_ERR_NO_BINS"
    assert b"sm_103a" in lib.ib_version()


def test_kernel_widths_on_host(abi):
    """3- and 6-point kernels: plans size their boxes for the width; compensated plans and batches reject them."""
    lib = abi.load()
    size = ctypes.c_size_t()
    sizes = {}
    for k in (abi.IB_KERNEL_PESKIN4, abi.IB_KERNEL_ROMA3, abi.IB_KERNEL_BSPLINE6):
        assert lib.ib_plan_footprint(ctypes.byref(_desc(abi, kernel=k)), ctypes.byref(size)) == abi.IB_OK
        sizes[k] = size.value
    boxes = {k: 4096 * 3 * (8 + w) ** 3 * 4 for k, w in ((0, 4), (2, 3), (3, 6))}
    assert sizes[2] - sizes[0] == pytest.approx(boxes[2] - boxes[0], abs=4096)
    assert sizes[3] - sizes[0] == pytest.approx(boxes[3] - boxes[0], abs=4096)
    h = ctypes.c_void_p()
    for k in (abi.IB_KERNEL_ROMA3, abi.IB_KERNEL_BSPLINE6):
        d = _desc(abi, kernel=k, flags=abi.IB_PLAN_COMPENSATED)
        assert lib.ib_plan_footprint(ctypes.byref(d), ctypes.byref(size)) == abi.IB_ERR_INVALID_ARG
        assert lib.ib_plan_create(ctypes.byref(d), ctypes.byref(h)) == abi.IB_ERR_INVALID_ARG
        b = abi.ib_batch_desc()
        b.dim, b.grid, b.kernel, b.dtype, b.ncomp = 3, abi.IB_GRID_MAC, k, abi.IB_F32, 3
        b.max_jobs, b.max_points, b.max_cells, b.max_tiles = 4, 1000, 1 << 16, 256
        assert lib.ib_batch_footprint(ctypes.byref(b), ctypes.byref(size)) == abi.IB_ERR_INVALID_ARG
        assert lib.ib_interpolate_noalloc(ctypes.byref(_desc(abi, kernel=k)), 0, None, None, None, None) == \
            abi.IB_ERR_INVALID_ARG
    assert lib.ib_plan_footprint(ctypes.byref(_desc(abi, kernel=4)), ctypes.byref(size)) == abi.IB_ERR_INVALID_ARG


def test_bounded_flags_on_host(abi):
    """Bounded dimensions: accepted per dimension (z only in 3-D); the scratch grows by the extended grid."""
    lib = abi.load()
    size = ctypes.c_size_t()
    assert lib.ib_plan_footprint(ctypes.byref(_desc(abi)), ctypes.byref(size)) == abi.IB_OK
    base = size.value
    d = _desc(abi, flags=abi.IB_PLAN_BOUNDED_Z)
    assert lib.ib_plan_footprint(ctypes.byref(d), ctypes.byref(size)) == abi.IB_OK
    # 128 x 128 x 136 extended cells: boxes of 16 x 16 x 17 tiles, an extended grid of 3 components
    assert size.value > base + 3 * 128 * 128 * 136 * 4
    d2 = _desc(abi, dim=2, n=(64, 64), ncomp=2, flags=abi.IB_PLAN_BOUNDED_Z)
    assert lib.ib_plan_footprint(ctypes.byref(d2), ctypes.byref(size)) == abi.IB_ERR_INVALID_ARG
    d3 = _desc(abi, dim=2, n=(64, 64), ncomp=2, flags=abi.IB_PLAN_BOUNDED_X | abi.IB_PLAN_BOUNDED_Y)
    assert lib.ib_plan_footprint(ctypes.byref(d3), ctypes.byref(size)) == abi.IB_OK


def test_stokes_validation_on_host(abi):
    """ib_stokes_create rejects what it cannot solve before any CUDA or cuFFT call."""
    lib = abi.load()
    h = ctypes.c_void_p(7)
    bad = [dict(grid=abi.IB_GRID_CELL_CENTERED), dict(ncomp=2), dict(dim=4), dict(n=(1, 8, 8)), dict(n=(8, 8, 0)),
           dict(L=(1.0, 0.0, 1.0)), dict(L=(1.0, float("inf"), 1.0)), dict(dtype=3), dict(n=(2048, 2048, 1024))]
    for kw in bad:
        assert lib.ib_stokes_create(ctypes.byref(_desc(abi, **kw)), ctypes.byref(h)) == abi.IB_ERR_INVALID_ARG, kw
        assert h.value is None
        h = ctypes.c_void_p(7)
    assert lib.ib_stokes_create(None, ctypes.byref(h)) == abi.IB_ERR_INVALID_ARG
    assert lib.ib_stokes_solve(None, None, None, None, 1.0, 1.0, None) == abi.IB_ERR_INVALID_ARG
    assert lib.ib_stokes_destroy(None) == abi.IB_OK


def test_batch_footprints_on_host(abi):
    lib = abi.load()
    d = abi.ib_batch_desc(dim=3, grid=abi.IB_GRID_MAC, kernel=0, dtype=0, ncomp=3, max_jobs=64,
                          max_points=1 << 20, max_cells=1 << 24, max_tiles=8192, flags=0)
    size = ctypes.c_size_t()
    assert lib.ib_batch_footprint(ctypes.byref(d), ctypes.byref(size)) == abi.IB_OK
    job = abi.ib_job()
    for b, v in enumerate((96, 96, 96)):
        job.n[b] = v
        job.L[b] = 1.0
    job.npts = 5000
    jb = ctypes.c_size_t()
    tiles = ctypes.c_longlong()
    assert lib.ib_batch_job_footprint(ctypes.byref(d), ctypes.byref(job), ctypes.byref(jb), ctypes.byref(tiles)) == 0
    assert tiles.value == 12 ** 3                 # 96 / 8 tiles per dimension
    assert jb.value == 4 * (96 ** 3 + 4 * 5000) + 12 ** 3 * 3 * 12 ** 3 * 4
    d.max_cells = 0
    assert lib.ib_batch_footprint(ctypes.byref(d), ctypes.byref(size)) == abi.IB_ERR_INVALID_ARG


def test_wave_admission_is_fifo_and_respects_caps_and_budget():
    from paper_2012_06646_gb300.serve import WaveCaps, admit_wave
    caps = WaveCaps(jobs=3, points=1000, cells=10 ** 6, tiles=100)
    q = [(100, 1000, 10, 1)] * 5
    assert admit_wave(q, caps, inflight=0, budget=10 ** 9) == (3, 30)          # job cap
    assert admit_wave(q, caps, inflight=0, budget=25) == (2, 20)               # budget
    assert admit_wave(q, caps, inflight=20, budget=25) == (0, 0)               # budget already used
    assert admit_wave([(2000, 1, 10, 1)], caps, inflight=0, budget=10 ** 9) == (0, 0)   # over the point cap
    assert admit_wave([(10, 1, 10 ** 10, 1)], caps, inflight=0, budget=5) == (1, 10 ** 10)  # alone: runs anyway
    big_first = [(900, 1, 1, 1), (200, 1, 1, 1), (50, 1, 1, 1)]
    assert admit_wave(big_first, caps, 0, 10 ** 9) == (1, 1)                   # FIFO: no overtaking


def test_jobs_that_never_fit_a_slot_are_named():
    from paper_2012_06646_gb300.serve import WaveCaps, never_fits
    caps = WaveCaps(jobs=4, points=1000, cells=4096, tiles=64)
    assert never_fits(1000, 4096, 64, caps) == ""
    assert "points" in never_fits(1001, 8, 1, caps)
    assert "cells" in never_fits(10, 4097, 1, caps)
    assert "tiles" in never_fits(10, 8, 65, caps)


def test_allocator_pair_checks_on_host(abi):
    # ib_set_allocator makes no CUDA call: both NULL restores cudaMalloc, one NULL is an error.
    lib = abi.load()
    null_a, null_f = abi.ib_alloc_fn(), abi.ib_free_fn()
    calls = []
    a = abi.ib_alloc_fn(lambda n, c: calls.append(n) or 0)
    f = abi.ib_free_fn(lambda p, c: calls.append(p))
    assert lib.ib_set_allocator(a, null_f, None) == abi.IB_ERR_INVALID_ARG
    assert lib.ib_set_allocator(null_a, f, None) == abi.IB_ERR_INVALID_ARG
    assert lib.ib_set_allocator(a, f, None) == abi.IB_OK
    assert lib.ib_set_allocator(null_a, null_f, None) == abi.IB_OK
    assert calls == []                            # installing a pair allocates nothing
    from paper_2012_06646_gb300 import plan
    with pytest.raises(ValueError):
        plan.set_allocator(lambda n: 0, None)
    plan.set_allocator(lambda n: 0, lambda p: None)
    assert plan._allocator is not None
    plan.set_allocator()
    assert plan._allocator is None


def test_inputs_are_deterministic_and_stream_separated():
    import numpy as np
    import ib_inputs
    a = ib_inputs.uniform_points(3, 100, (1.0, 2.0, 3.0), 3)
    b = ib_inputs.uniform_points(3, 100, (1.0, 2.0, 3.0), 3)
    c = ib_inputs.uniform_points(4, 100, (1.0, 2.0, 3.0), 3)
    assert np.array_equal(a, b) and not np.array_equal(a, c)
    assert a.dtype == np.float32 and np.all(a >= 0) and np.all(a < np.array([1.0, 2.0, 3.0], np.float32))
    g = ib_inputs.normal_array(1, (20000,), dtype=np.float64)
    assert abs(g.mean()) < 0.03 and abs(g.std() - 1.0) < 0.03
    assert len(ib_inputs.icosphere(4)) == 2562
    assert abs(ib_inputs.rbc_volume(3.91) - 94.4) < 0.2
    # the cheap large-case generators: deterministic, in range, and not degenerate
    u1 = ib_inputs.uniform_array(5, (30000, 3))
    assert np.array_equal(u1, ib_inputs.uniform_array(5, (30000, 3)))
    assert u1.dtype == np.float32 and u1.min() >= -1.0 and u1.max() < 1.0 and abs(float(u1.mean())) < 0.02
    w = ib_inputs.wave_field(16)
    assert w.shape == (3, 16, 16, 16) and w.dtype == np.float32 and np.abs(w).max() <= 1.0
    assert np.array_equal(w, ib_inputs.wave_field(16))
    assert np.abs(np.diff(w, axis=3)).mean() > 0.5           # neighbouring nodes differ strongly
    k, l, m, ph = 3, 251, 17, 0.3                             # component 0 at node (x, y, z) = (1, 2, 3)
    assert abs(float(w[0, 3, 2, 1]) - np.sin(2 * np.pi * (k * 1 + l * 2 + m * 3) / 16 + ph)) < 1e-6


def test_membrane_packing_reaches_the_stated_density_without_overlap():
    """The clustered-membrane workload: 17 randomly oriented red cells (R0 = 3.91/16
    of the box) compressed to about 40 % volume fraction; no point of a fine
    (subdivision-5) surface of one cell lies inside another, over periodic
    images; the paper's 8832 points per cell gives the denser variant."""
    import numpy as np
    import ib_inputs
    m = ib_inputs.pack_membranes(0)
    assert len(m.centres) == 17 and len(m.X) == 17 * 2562
    assert 0.385 < m.volume_fraction < 0.40
    assert m.X.dtype == np.float32 and m.X.min() >= 0.0 and m.X.max() < 1.0
    P = ib_inputs.rbc_points(m.R0, ib_inputs.icosphere(5))
    for i in range(17):
        for j in range(17):
            if i != j:
                d = m.centres[i] - m.centres[j]
                d -= np.round(d)
                assert not ib_inputs.rbc_inside((P @ m.rotations[i].T + d) @ m.rotations[j], m.R0).any()
    # orientations are rotations (orthonormal, det 1)
    for R in m.rotations:
        assert np.allclose(R @ R.T, np.eye(3), atol=1e-9) and abs(np.linalg.det(R) - 1.0) < 1e-9
    m2 = ib_inputs.pack_membranes(0)
    assert np.array_equal(m.X, m2.X)                                  # depends on the seed only
    d8 = ib_inputs.pack_membranes(1, points_per_cell=8832)
    assert len(d8.centres) == 17 and len(d8.X) == 17 * 8832
    sph = ib_inputs.fibonacci_sphere(8832)
    assert np.allclose(np.linalg.norm(sph, axis=1), 1.0) and abs(sph.mean(axis=0)).max() < 1e-3
