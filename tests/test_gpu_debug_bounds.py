"""The IB_DEBUG_BOUNDS build: every computed index of the kernels checked on
the device (a failure skips the access and is reported as IB_ERR_BOUNDS).
Runs the cases of _debug_cases.py on that build in a child process: no check
may fail, and every output must be bit-identical to the release build's."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


def test_debug_bounds_build_passes_and_matches_release():
    from paper_2012_06646_gb300 import build
    from paper_2012_06646_gb300.build import build as build_lib
    build()
    build_lib(debug_bounds=True)
    import _debug_cases
    release = _debug_cases.run_cases()
    assert "IB_DEBUG_BOUNDS" not in release["version"]
    env = dict(os.environ, IBGB_DEBUG_BOUNDS="1", PYTHONPATH=os.pathsep.join([ROOT, HERE]))
    res = subprocess.run([sys.executable, os.path.join(HERE, "_debug_cases.py")], capture_output=True, text=True,
                         env=env, cwd=ROOT, timeout=600)
    assert res.returncode == 0, res.stderr[-3000:]
    debug = json.loads(res.stdout.strip().splitlines()[-1])
    assert "IB_DEBUG_BOUNDS" in debug.pop("version")
    release.pop("version")
    assert debug.keys() == release.keys()
    diff = [k for k in release if release[k] != debug[k]]
    assert not diff, f"debug build differs from release on {diff}"
