"""The allocation-free <Z_q>/norm entry point (for callers that cannot call cudaMalloc,
such as hosts whose device memory is owned by their own pool allocator).

It is called through the C ABI and compared with the allocating entry point
qs_expectation_z on the same state, twice in a row (its static scratch keeps the previous
call's contents, which must not leak into the next result).  This file sorts last so that
a run stopping at the first failure has already run every other test."""
import numpy as np
import pytest

from paper_2409_14697_gb300 import inputs
from tests.gpu_util import require_gpu

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("dtype", [2, 1])
@pytest.mark.parametrize("n", [3, 12, 23])
def test_noalloc_expz_matches_allocating_entry_point(n, dtype):
    require_gpu()
    from paper_2409_14697_gb300 import qs
    qs.load()
    h = qs.qs_create(n, dtype)
    try:
        psi = inputs.gaussian_state(n, seed=300 + n) * 1.3
        qs.qs_set_amplitudes(h, psi.astype(np.complex64 if dtype == 1 else np.complex128))
        ez_ref, nrm_ref = qs.qs_expectation_z(h)
        dev_ptr = qs.qs_info(h)[2]
        for _ in range(2):
            ez, nrm = qs.qs_expectation_z_noalloc(dev_ptr, n, dtype)
            # FP64 accumulation in both; only the block split (summation order) differs
            assert abs(nrm - nrm_ref) <= 1e-13 * nrm_ref
            assert np.max(np.abs(ez - ez_ref)) <= 1e-13 * nrm_ref
        # a second, different state through the same scratch
        qs.qs_apply_circuit(h, inputs.brickwork(n, 2, seed=n) if n >= 2 else [])
        ez_ref2, nrm_ref2 = qs.qs_expectation_z(h)
        ez2, nrm2 = qs.qs_expectation_z_noalloc(dev_ptr, n, dtype)
        assert abs(nrm2 - nrm_ref2) <= 1e-13 * nrm_ref2
        assert np.max(np.abs(ez2 - ez_ref2)) <= 1e-13 * nrm_ref2
    finally:
        qs.qs_destroy(h)


def test_noalloc_rejects_sizes_beyond_its_scratch():
    require_gpu()
    from paper_2409_14697_gb300 import qs
    h = qs.qs_create(4, 2)
    try:
        with pytest.raises(qs.QsError) as e:
            qs.qs_expectation_z_noalloc(qs.qs_info(h)[2], 33, 2)
        assert e.value.code == qs.QS_ERR_INVALID
    finally:
        qs.qs_destroy(h)
