"""GPU parity of the batched persistent launch (one graph-captured kernel for many
circuits of different widths) against the FP64 oracle, and its bounded-wait timeout."""
import numpy as np
import pytest

import oracle
from paper_2409_14697_gb300 import inputs
from tests.gpu_util import TOL_C128, TOL_C64, fidelity_gap, require_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def qs():
    require_gpu()
    from paper_2409_14697_gb300 import qs as q
    q.load()
    return q


@pytest.mark.parametrize("dtype", [1, 2])
def test_batch_matches_oracle(qs, dtype):
    circs = inputs.batched_circuits(48, seed=3, n_range=(6, 17), depth_range=(2, 12))
    circs.append((14, inputs.qaoa_3regular(14, p=2)))
    circs.append((16, inputs.qft(16)))
    b = qs.qs_batch_create(circs, dtype, qs.options(chunk_m=12 if dtype == 2 else 13))
    try:
        info = qs.qs_batch_info(b)
        assert info["circuits"] == len(circs)
        for rep in range(2):           # replaying the graph gives the same states
            qs.qs_batch_run(b)
            qs.qs_batch_synchronize(b)
            for i, (n, gates) in enumerate(circs):
                got = qs.qs_batch_amplitudes(b, i, n, dtype).astype(np.complex128)
                want = oracle.run(oracle.zero_state(n), n, gates)
                err = np.max(np.abs(got - want))
                assert err <= (TOL_C128 if dtype == 2 else TOL_C64), (i, n, err)
                if dtype == 1:
                    assert fidelity_gap(got, want) <= 1e-6
    finally:
        qs.qs_batch_destroy(b)


def test_batch_multi_pass_small_tiles(qs):
    """Force many passes per circuit (tile of 2^8) so the cross-CTA pass dependencies
    are exercised heavily."""
    circs = inputs.batched_circuits(24, seed=5, n_range=(10, 16), depth_range=(4, 10))
    b = qs.qs_batch_create(circs, 1, qs.options(chunk_m=8))
    try:
        assert qs.qs_batch_info(b)["passes"] > 3 * len(circs)
        qs.qs_batch_run(b)
        qs.qs_batch_synchronize(b)
        for i, (n, gates) in enumerate(circs):
            got = qs.qs_batch_amplitudes(b, i, n, 1).astype(np.complex128)
            want = oracle.run(oracle.zero_state(n), n, gates)
            assert np.max(np.abs(got - want)) <= TOL_C64
    finally:
        qs.qs_batch_destroy(b)


def test_batch_wait_times_out_and_context_survives(qs):
    """A dependency that nothing satisfies (test hook) must end in QS_ERR_TIMEOUT after
    the short wait limit, not hang; the GPU stays usable afterwards."""
    circs = inputs.batched_circuits(8, seed=7, n_range=(14, 15), depth_range=(3, 4))
    o = qs.options(chunk_m=10)
    o.reserved[0] = 200000      # 0.2 s
    o.reserved[1] = 1           # unsatisfiable dependency
    b = qs.qs_batch_create(circs, 1, o)
    try:
        qs.qs_batch_run(b)
        with pytest.raises(qs.QsError) as e:
            qs.qs_batch_synchronize(b)
        assert e.value.code == qs.QS_ERR_TIMEOUT
    finally:
        qs.qs_batch_destroy(b)
    # the context is still healthy
    h = qs.qs_create(10, 2)
    try:
        qs.qs_apply_circuit(h, [("h", (q,), ()) for q in range(10)])
        assert abs(qs.qs_norm(h) - 1.0) < 1e-14
    finally:
        qs.qs_destroy(h)
