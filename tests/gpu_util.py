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


def _chunks(size, chunk=1 << 22):
    return [(lo, min(size, lo + chunk)) for lo in range(0, size, chunk)]


def _pool():
    import concurrent.futures as cf
    import os
    try:
        n = len(os.sched_getaffinity(0))
    except AttributeError:
        n = os.cpu_count() or 1
    return cf.ThreadPoolExecutor(max_workers=max(1, n))


def compare_large(got, want):
    """(max-abs error, 1 - fidelity) of a GPU result (complex64 or complex128) against the
    complex128 oracle state, computed in FP64 over chunks on every host core (numpy releases
    the GIL), for states too large for one numpy temporary."""
    assert got.size == want.size

    def part(r):
        lo, hi = r
        g = got[lo:hi].astype(np.complex128, copy=False)
        w = want[lo:hi]
        return (float(np.max(np.abs(g - w))), complex(np.vdot(w, g)),
                float(np.vdot(g, g).real), float(np.vdot(w, w).real))

    with _pool() as ex:
        parts = list(ex.map(part, _chunks(got.size)))
    err = max(p[0] for p in parts)
    ov = sum(p[1] for p in parts)
    ng = sum(p[2] for p in parts)
    nw = sum(p[3] for p in parts)
    return err, 1.0 - abs(ov) ** 2 / (ng * nw)
