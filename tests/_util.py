"""Shared helpers for the parity tests (no method arithmetic here)."""
import numpy as np


def block_err(got, ref):
    """Block-normwise relative error max|got - ref| / max|ref| (0 if both are 0)."""
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    scale = np.abs(ref).max() if ref.size else 0.0
    diff = np.abs(got - ref).max() if ref.size else 0.0
    if scale == 0.0:
        return diff
    return diff / scale


# Tolerances (stated per precision):
#   FP64 path: every block rel <= 1e-10.
#   FP32 Phi path: A, B-, B+, S rel <= 1e-4; state-derived defect / penalty rel <= 1e-10.
TOL_FP64 = 1e-10
TOL_FP32_PHI = 1e-4
