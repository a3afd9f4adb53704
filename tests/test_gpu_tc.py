"""GPU parity of the tensor-core fused-block path (K3: tcgen05 kind::tf32, 3xTF32 split
products, FP32 accumulation) for complex64 against the FP64 oracle."""
import numpy as np
import pytest

import oracle
from paper_2409_14697_gb300 import inputs
from tests.gpu_util import TOL_C64, fidelity_gap, require_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def qs():
    require_gpu()
    from paper_2409_14697_gb300 import qs as q
    q.load()
    return q


def run(qs, n, psi0, gates, **kw):
    h = qs.qs_create(n, 1)
    try:
        qs.qs_set_amplitudes(h, psi0.astype(np.complex64))
        qs.qs_apply_circuit(h, gates, qs.options(**kw))
        return qs.qs_amplitudes(h).astype(np.complex128), qs.qs_last_stats(h)
    finally:
        qs.qs_destroy(h)


@pytest.mark.parametrize("k", [4, 5, 6])
def test_single_dense_block_fused_mode(qs, k):
    """One random k-qubit unitary on scattered qubits, FUSED mode: one tensor-core pass."""
    n = 14
    r = np.random.default_rng(k)
    qubits = tuple(int(x) for x in r.choice(n, size=k, replace=False))
    gates = [("dense", qubits, inputs.random_unitary(k, seed=k))]
    psi0 = inputs.gaussian_state(n, seed=k)
    want = oracle.run(psi0.astype(np.complex64).astype(np.complex128), n, gates)
    got, st = run(qs, n, psi0, gates, mode=qs.QS_MODE_FUSED, fuse_k=k)
    assert st["passes"] == 1
    assert st["tc_blocks"] == 1          # the block ran on the tensor cores
    # 2^(n-k) groups x 2^(k+1) x 2^(k+1) multiply-adds, three TF32 products, 2 flops each
    assert st["tc_flops"] == 6.0 * 2.0 ** (n + k + 2)
    assert np.max(np.abs(got - want)) <= TOL_C64
    assert fidelity_gap(got, want) <= 1e-6


@pytest.mark.parametrize("fk", [4, 5, 6])
@pytest.mark.parametrize("n", [13, 16, 20])
def test_brickwork_auto_tensor_cores(qs, n, fk):
    gates = inputs.brickwork(n, 8, seed=n + fk)
    psi0 = oracle.zero_state(n)
    want = oracle.run(psi0.copy(), n, gates)
    got, st = run(qs, n, psi0, gates, fuse_k=fk)
    assert np.max(np.abs(got - want)) <= TOL_C64
    assert fidelity_gap(got, want) <= 1e-6
    assert st["ops_after_fuse"] < len(gates)
    assert st["tc_blocks"] > 0


@pytest.mark.parametrize("family", ["qaoa", "tfim", "random"])
def test_families_tensor_cores(qs, family):
    n = 18
    if family == "qaoa":
        gates = inputs.qaoa_3regular(n, p=4, seed=2)
    elif family == "tfim":
        gates = inputs.tfim(n, steps=10)
    else:
        gates = inputs.random_circuit(n, 300, seed=4)
    psi0 = inputs.gaussian_state(n, seed=6)
    want = oracle.run(psi0.astype(np.complex64).astype(np.complex128), n, gates)
    got, st = run(qs, n, psi0, gates, fuse_k=5)
    assert np.max(np.abs(got - want)) <= TOL_C64
    assert fidelity_gap(got, want) <= 1e-6
    assert st["tc_blocks"] > 0


def test_tensor_core_path_matches_simt_path_24q(qs):
    """The same circuit with fusion on the tensor cores (k = 6) and on SIMT (k = 2)."""
    n = 24
    gates = inputs.brickwork(n, 12, seed=9)
    psi0 = inputs.gaussian_state(n, seed=9)
    a, sa = run(qs, n, psi0, gates, fuse_k=6)
    b, sb = run(qs, n, psi0, gates, fuse_k=2)
    assert sa["tc_blocks"] > 0 and sb["tc_blocks"] == 0
    assert np.max(np.abs(a - b)) <= TOL_C64
    assert fidelity_gap(a, b) <= 1e-6
