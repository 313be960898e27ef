"""Helpers for the GPU parity tests: device transfer and the tolerance checks.

Tolerances (the accuracy target of the FP32 path):
  spreading      per node   |f - f_ref| <= 1e-5 * fabs_k + floor, and f = 0 exactly where fabs_k = 0
  interpolation  per point  |U - U_ref| <= 1e-5 * Uabs_j + floor, and max |U - U_ref| <= 1e-5 max |U_ref|
where fabs_k / Uabs_j are the oracle's sums of |contribution|.  `floor` is
64 FLT_MIN: single contributions below the FP32 normal range may flush to
zero and are not representable in FP32 anyway.  FP64 plans use 1e-12.
"""
import numpy as np
import torch

FLOOR32 = 64 * float(np.finfo(np.float32).tiny)
FLOOR64 = 64 * float(np.finfo(np.float64).tiny)


def dev(a, device="cuda"):
    return torch.from_numpy(np.ascontiguousarray(a)).to(device)


def host(t):
    torch.cuda.synchronize()
    return t.detach().cpu().numpy()


def assert_spread_close(f, f_ref, fabs, rel=1e-5, floor=FLOOR32, what="spread"):
    f = np.asarray(f, dtype=np.float64)
    err = np.abs(f - f_ref)
    bad = err > rel * fabs + floor
    if bad.any():
        i = np.argmax(err / (fabs + floor))
        raise AssertionError(f"{what}: {int(bad.sum())} nodes out of tolerance; worst rel "
                             f"{float((err / (fabs + floor)).ravel()[i]):.3e} (got {f.ravel()[i]!r}, "
                             f"want {f_ref.ravel()[i]!r}, fabs {fabs.ravel()[i]!r})")
    assert np.all(f[fabs == 0] == 0), f"{what}: nonzero value where no point contributes"


def assert_interp_close(U, U_ref, Uabs, rel=1e-5, floor=FLOOR32, what="interp"):
    U = np.asarray(U, dtype=np.float64)
    err = np.abs(U - U_ref)
    bad = err > rel * Uabs + floor
    if bad.any():
        i = np.argmax(err / (Uabs + floor))
        raise AssertionError(f"{what}: {int(bad.sum())} values out of tolerance; worst rel "
                             f"{float((err / (Uabs + floor)).ravel()[i]):.3e}")
    if U_ref.size:
        assert err.max() <= rel * max(np.abs(U_ref).max(), floor) + floor, f"{what}: max error too large"
