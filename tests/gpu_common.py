"""Helpers shared by the GPU parity tests (no solver arithmetic here)."""
import numpy as np

TOL64 = 1e-12   # relative, FP64 kernels
TOL32 = 1e-5    # relative, FP32 kernels


def rel(a, b) -> float:
    """max |a - b| / max |b|."""
    den = np.abs(b).max()
    return float(np.abs(a - b).max() / (den if den > 0 else 1.0))


def lib_built():
    from paper_1011_2775_gb300 import build
    return build.build()
