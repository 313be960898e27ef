"""Build the CUDA library in-tree: paper_2012_06646_gb300/_lib/libibgb.so.

Each translation unit under csrc/ is compiled by nvcc for sm_103a only, in
parallel, then linked into one shared library (CUDA runtime linked
statically).  The library exports exactly the C ABI of include/ib.h.
build(debug_bounds=True) builds the same sources with IB_DEBUG_BOUNDS (every
kernel's computed indices checked, failures reported as IB_ERR_BOUNDS) into
_lib_debug/libibgb.so, which _abi loads when IBGB_DEBUG_BOUNDS=1.
"""

from __future__ import annotations

import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
LIBDIR = os.path.join(HERE, "_lib")
SO = os.path.join(LIBDIR, "libibgb.so")
LIBDIR_DEBUG = os.path.join(HERE, "_lib_debug")
SOURCES = ["ib_bin.cu", "ib_ops.cu", "ib_width.cu", "ib_bounds.cu", "ib_paper.cu", "ib_fluid.cu", "ib_api.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    path = shutil.which("nvcc")
    if path:
        return path
    cand = "/usr/local/cuda/bin/nvcc"
    if os.path.exists(cand):
        return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libibgb.so")


def _stale(so: str = SO) -> bool:
    if not os.path.exists(so):
        return True
    so_time = os.path.getmtime(so)
    deps = [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [os.path.join(ROOT, "include", "ib.h"), __file__]
    return any(os.path.getmtime(d) > so_time for d in deps)


def build(force: bool = False, verbose: bool = False, ptxas_info: bool = False, debug_bounds: bool = False) -> str:
    libdir = LIBDIR_DEBUG if debug_bounds else LIBDIR
    so = os.path.join(libdir, "libibgb.so")
    if not force and not _stale(so):
        return so
    os.makedirs(libdir, exist_ok=True)
    cc = nvcc()
    common = [cc, "-O3", "-std=c++17", *ARCH, "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
              "-I", os.path.join(ROOT, "include")]
    if debug_bounds:
        common.append("-DIB_DEBUG_BOUNDS")
    if ptxas_info:
        common += ["-Xptxas", "-v"]
    objs = []

    def compile_one(src: str) -> str:
        obj = os.path.join(libdir, src.replace(".cu", ".o"))
        cmd = common + ["-c", os.path.join(CSRC, src), "-o", obj]
        res = subprocess.run(cmd, capture_output=True, text=True)
        if res.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src}:\n{res.stdout}\n{res.stderr}")
        if verbose or ptxas_info:
            sys.stderr.write(res.stdout + res.stderr)
        return obj

    with ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(compile_one, SOURCES))
    tmp = so + f".tmp{os.getpid()}"
    # cuFFT (the Stokes solve) is linked dynamically, found through the
    # toolkit's library directory when the loader path lacks it.
    cudalib = os.path.join(os.path.dirname(os.path.dirname(os.path.realpath(cc))), "lib64")
    # Only the C ABI (ib_*) is exported (linker version script).
    exports = os.path.join(CSRC, "libibgb.map")
    res = subprocess.run([cc, "-shared", *ARCH, "-o", tmp, *objs, "-lcufft", "-Xlinker", f"-rpath={cudalib}",
                          "-Xlinker", f"--version-script={exports}"],
                         capture_output=True, text=True)
    if res.returncode != 0:
        raise RuntimeError(f"nvcc link failed:\n{res.stdout}\n{res.stderr}")
    os.replace(tmp, so)
    return so


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True, ptxas_info="--ptxas" in sys.argv,
                debug_bounds="--debug-bounds" in sys.argv))
