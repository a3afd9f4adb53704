"""Helpers shared by the GPU parity tests (no simulation arithmetic here)."""
import numpy as np
import pytest

# Tolerances.  complex128: the target of 1e-12 max-abs against the FP64 oracle.
# complex64: FP32 storage has unit roundoff 2^-24 ~ 6e-8 per operation; a gate touches
# each amplitude with <= 8 operations, so after g gates the error grows like
# 6e-8 * 8 * sqrt(g) * max|a|; 2e-5 covers g <= 400 at max|a| <= 1 with margin.
TOL_C128 = 1e-12
TOL_C64 = 2e-5


def require_gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def fidelity_gap(a, b):
    a = np.asarray(a, dtype=np.complex128)
    b = np.asarray(b, dtype=np.complex128)
    ov = abs(np.vdot(a, b)) ** 2
    return 1.0 - ov / (np.vdot(a, a).real * np.vdot(b, b).real)
