"""GPU edge cases: empty circuits, the smallest states on every path, k = 2^n top-K, the
largest complex64 state this GPU holds, and clean failure when a state cannot fit."""
import numpy as np
import pytest

import oracle
from paper_2409_14697_gb300 import inputs
from tests.gpu_util import TOL_C128, TOL_C64, require_gpu

pytestmark = pytest.mark.gpu

MODES = ["gate", "auto", "chunk", "fused"]


@pytest.fixture(scope="module")
def qs():
    require_gpu()
    from paper_2409_14697_gb300 import qs as q
    q.load()
    return q


def mode_id(qs, name):
    return {"gate": qs.QS_MODE_GATE, "auto": qs.QS_MODE_AUTO, "chunk": qs.QS_MODE_CHUNK,
            "fused": qs.QS_MODE_FUSED}[name]


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("dtype", [2, 1])
def test_empty_circuit_leaves_state(qs, mode, dtype):
    n = 9
    psi0 = inputs.gaussian_state(n, seed=1).astype(np.complex128 if dtype == 2 else np.complex64)
    h = qs.qs_create(n, dtype)
    try:
        qs.qs_set_amplitudes(h, psi0)
        qs.qs_apply_circuit(h, [], qs.options(mode=mode_id(qs, mode)))
        assert np.array_equal(qs.qs_amplitudes(h), psi0)
    finally:
        qs.qs_destroy(h)


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("dtype", [2, 1])
@pytest.mark.parametrize("n", [1, 2, 4])
def test_smallest_states_every_path(qs, mode, dtype, n):
    gates = inputs.random_circuit(n, 60, seed=n)
    if n >= 2:
        gates.append(("dense", tuple(range(n))[:2], inputs.random_unitary(2, seed=n)))
    psi0 = inputs.gaussian_state(n, seed=n)
    want = oracle.run(psi0.copy(), n, gates)
    h = qs.qs_create(n, dtype)
    try:
        qs.qs_set_amplitudes(h, psi0.astype(np.complex128 if dtype == 2 else np.complex64))
        qs.qs_apply_circuit(h, gates, qs.options(mode=mode_id(qs, mode), fuse_k=2))
        got = qs.qs_amplitudes(h).astype(np.complex128)
        ez, nrm = qs.qs_expectation_z(h)
        idx, amp = qs.qs_top_amplitudes(h, 1 << n)
    finally:
        qs.qs_destroy(h)
    tol = TOL_C128 if dtype == 2 else TOL_C64
    assert np.max(np.abs(got - want)) <= tol
    assert np.max(np.abs(ez - oracle.expz(got, n))) <= 1e-13
    assert sorted(idx.tolist()) == list(range(1 << n))     # k = 2^n returns everything


def test_largest_complex64_state(qs):
    """34 qubits complex64 = 128 GiB on one GPU: a sweep, its inverse and the norm."""
    n = 34
    h = qs.qs_create(n, 1)
    try:
        gates = [("h", (q,), ()) for q in range(n)] + inputs.gate_sweep(n, "u3", count=n) + \
            inputs.gate_sweep(n, "cnot", count=n)
        qs.qs_apply_circuit(h, gates + inputs.inverse(gates), qs.options(mode=qs.QS_MODE_GATE))
        a = qs.qs_amplitudes(h, 0, 4)
        assert abs(qs.qs_norm(h) - 1.0) < 1e-5
        assert abs(a[0] - 1.0) < 1e-4 and np.max(np.abs(a[1:])) < 1e-4
    finally:
        qs.qs_destroy(h)


def test_state_that_cannot_fit(qs):
    with pytest.raises(qs.QsError) as e:
        qs.qs_create(36, 2)          # 1 TiB
    assert e.value.code == qs.QS_ERR_NOMEM
    h = qs.qs_create(10, 2)          # and the device is still usable
    qs.qs_destroy(h)
