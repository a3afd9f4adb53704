"""The allocation-free <Z_q>/norm entry point (for callers that cannot call cudaMalloc,
such as hosts whose device memory is owned by their own pool allocator).

It is called through the C ABI and compared with the allocating entry point
qs_expectation_z on the same state, twice in a row (its static scratch keeps the previous
call's contents, which must not leak into the next result), and with the oracle's norm
and <Z_q>.  Up to 30 qubits both entry points split the state into the same blocks, so
their results must agree bit for bit; at 31 and 32 qubits the allocation-free one uses
larger blocks (at most 2^14 of them fit its scratch), and there the closed form of
H^n|0> pins it.  This file sorts last so that a run stopping at the first failure has
already run every other test."""
import numpy as np
import pytest

import oracle
from paper_2409_14697_gb300 import inputs
from tests.gpu_util import require_gpu

pytestmark = pytest.mark.gpu


def _qs():
    require_gpu()
    from paper_2409_14697_gb300 import qs
    qs.load()
    return qs


@pytest.mark.parametrize("dtype", [2, 1])
@pytest.mark.parametrize("n", [3, 12, 23])
def test_noalloc_expz_matches_allocating_entry_point(n, dtype):
    qs = _qs()
    npdt = np.complex64 if dtype == 1 else np.complex128
    h = qs.qs_create(n, dtype)
    try:
        psi = (inputs.gaussian_state(n, seed=300 + n) * 1.3).astype(npdt)
        qs.qs_set_amplitudes(h, psi)
        ez_ref, nrm_ref = qs.qs_expectation_z(h)
        dev_ptr = qs.qs_info(h)[2]
        wide = psi.astype(np.complex128)
        want_ez, want_nrm = oracle.expz(wide, n), oracle.norm(wide, n)
        for _ in range(2):
            ez, nrm = qs.qs_expectation_z_noalloc(dev_ptr, n, dtype)
            # same blocks, same kernels, same order: the same bits
            assert nrm == nrm_ref
            assert np.array_equal(ez, ez_ref)
            # and the oracle's pairwise FP64 sums (a different summation order)
            assert abs(nrm - want_nrm) <= 1e-13 * want_nrm
            assert np.max(np.abs(ez - want_ez)) <= 1e-13 * want_nrm
        # a second, different state through the same scratch
        qs.qs_apply_circuit(h, inputs.brickwork(n, 2, seed=n))
        ez_ref2, nrm_ref2 = qs.qs_expectation_z(h)
        ez2, nrm2 = qs.qs_expectation_z_noalloc(dev_ptr, n, dtype)
        assert nrm2 == nrm_ref2
        assert np.array_equal(ez2, ez_ref2)
        now = qs.qs_amplitudes(h).astype(np.complex128)
        assert abs(nrm2 - oracle.norm(now, n)) <= 1e-13 * nrm2
        assert np.max(np.abs(ez2 - oracle.expz(now, n))) <= 1e-13 * nrm2
    finally:
        qs.qs_destroy(h)


@pytest.mark.parametrize("n", [31, 32])
def test_noalloc_block_split_beyond_30_qubits(n):
    """complex64 H^n|0> at 31 and 32 qubits (16 and 32 GiB): here the allocation-free entry
    point splits the state into 2^14 blocks of 2^(n-14) amplitudes, unlike the allocating
    one.  Every amplitude is the same real value v, so <Z_q> = 0 and the squared norm is
    2^n v^2, both exact in FP64 for any balanced summation tree."""
    qs = _qs()
    h = qs.qs_create(n, 1)
    try:
        qs.qs_apply_circuit(h, [("h", (q,), ()) for q in range(n)], qs.options(mode=qs.QS_MODE_GATE))
        head = qs.qs_amplitudes(h, 0, 4).astype(np.complex128)
        tail = qs.qs_amplitudes(h, (1 << n) - 4, 4).astype(np.complex128)
        v = head[0].real
        assert np.all(head == v) and np.all(tail == v)
        want_nrm = float(1 << n) * v * v
        ez_ref, nrm_ref = qs.qs_expectation_z(h)
        dev_ptr = qs.qs_info(h)[2]
        for _ in range(2):
            ez, nrm = qs.qs_expectation_z_noalloc(dev_ptr, n, 1)
            assert abs(nrm - want_nrm) <= 1e-15 * want_nrm, (nrm, want_nrm)
            assert np.max(np.abs(ez)) <= 1e-15, np.max(np.abs(ez))
            assert abs(nrm - nrm_ref) <= 1e-13 * nrm_ref
            assert np.max(np.abs(ez - ez_ref)) <= 1e-13 * nrm_ref
    finally:
        qs.qs_destroy(h)


def test_noalloc_rejects_sizes_beyond_its_scratch():
    qs = _qs()
    h = qs.qs_create(4, 2)
    try:
        with pytest.raises(qs.QsError) as e:
            qs.qs_expectation_z_noalloc(qs.qs_info(h)[2], 33, 2)
        assert e.value.code == qs.QS_ERR_INVALID
    finally:
        qs.qs_destroy(h)
