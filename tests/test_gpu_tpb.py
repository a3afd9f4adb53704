"""GPU parity of the Tensor Product Booster (QueenV2 Sec. III-A tier 1): on a state that
holds |0...0>, the prefix whose gates keep the qubits in independent groups is built as the
tensor product of the groups' sub-states in one write pass.  Results through the C ABI are
compared with the oracle (which applies every gate to the full vector) and with the same
call under QS_OPT_NO_TPB; qs_stats tells whether the booster ran."""
import math

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


def run(qs, n, dtype, gates, flags=0, fuse_k=0, h=None):
    own = h is None
    if own:
        h = qs.qs_create(n, dtype)
    try:
        qs.qs_apply_circuit(h, gates, qs.options(flags=flags, fuse_k=fuse_k))
        return qs.qs_amplitudes(h).astype(np.complex128), qs.qs_last_stats(h)
    finally:
        if own:
            qs.qs_destroy(h)


def tol(dtype):
    return TOL_C128 if dtype == 2 else TOL_C64


@pytest.mark.parametrize("dtype", [2, 1])
def test_hadamard_layer_is_one_write_pass(qs, dtype):
    """H on every qubit of |0...0> (the paper's Hadamard benchmark): one write pass."""
    n = 24
    gates = [("h", (q,), ()) for q in range(n)]
    got, st = run(qs, n, dtype, gates)
    assert st["tpb_gates"] == n and st["passes"] == 1
    want = oracle.run(oracle.zero_state(n), n, gates)
    assert np.max(np.abs(got - want)) <= tol(dtype)


@pytest.mark.parametrize("dtype", [2, 1])
@pytest.mark.parametrize("family", ["brickwork", "qft", "random"])
def test_circuits_from_zero_state_vs_oracle(qs, family, dtype):
    n = 22
    if family == "brickwork":
        gates = inputs.brickwork(n, 12, seed=5)
    elif family == "qft":
        gates = [("u3", (q,), (0.3 * q, 0.1, 0.2)) for q in range(n)] + inputs.qft(n)
    else:
        gates = [("h", (q,), ()) for q in range(n)] + inputs.random_circuit(n, 200, seed=6)
    want = oracle.run(oracle.zero_state(n), n, gates)
    got, st = run(qs, n, dtype, gates)
    off, st_off = run(qs, n, dtype, gates, flags=qs.QS_OPT_NO_TPB)
    assert st_off["tpb_gates"] == 0
    assert np.max(np.abs(got - want)) <= tol(dtype)
    assert np.max(np.abs(off - want)) <= tol(dtype)
    if dtype == 1:
        assert fidelity_gap(got, want) <= 1e-6
    if family != "qft":
        assert st["tpb_gates"] > 0 and st["passes"] <= st_off["passes"]


def test_three_groups(qs):
    """Components of 9 qubits (GHZ-like chains after a U3 layer) pack into three groups of
    the product pass (at most 17 qubits each)."""
    n = 27
    r = np.random.default_rng(3)
    gates = [("u3", (q,), tuple(r.uniform(0, 2 * math.pi, 3))) for q in range(n)]
    for b in (0, 9, 18):
        gates += [("cnot", (q, q + 1), ()) for q in range(b, b + 8)]
    gates += inputs.brickwork(n, 2, seed=4)
    want = oracle.run(oracle.zero_state(n), n, gates)
    got, st = run(qs, n, 1, gates)
    assert st["tpb_gates"] >= n + 24
    assert np.max(np.abs(got - want)) <= TOL_C64
    assert fidelity_gap(got, want) <= 1e-6


def test_only_from_a_known_zero_state(qs):
    """The booster runs only on |0...0>: after qs_create and qs_reset, not after amplitudes
    were written or another circuit ran."""
    n = 21
    gates = [("h", (q,), ()) for q in range(n)] + inputs.brickwork(n, 2, seed=8)
    h = qs.qs_create(n, 2)
    try:
        a, st = run(qs, n, 2, gates, h=h)
        assert st["tpb_gates"] > 0
        b, st = run(qs, n, 2, inputs.inverse(gates), h=h)     # the state is not |0> now
        assert st["tpb_gates"] == 0
        assert abs(b[0] - 1.0) <= 1e-12 and np.max(np.abs(b[1:])) <= 1e-12
        qs.qs_reset(h)
        c, st = run(qs, n, 2, gates, h=h)
        assert st["tpb_gates"] > 0 and np.array_equal(a, c)
        psi = inputs.gaussian_state(n, seed=2)
        qs.qs_set_amplitudes(h, psi)                         # written from the host
        d, st = run(qs, n, 2, gates, h=h)
        assert st["tpb_gates"] == 0
        want = oracle.run(psi.copy(), n, gates)
        assert np.max(np.abs(d - want)) <= TOL_C128
    finally:
        qs.qs_destroy(h)


def test_tensor_core_blocks_after_the_booster(qs):
    n = 22
    gates = inputs.brickwork(n, 10, seed=7)
    want = oracle.run(oracle.zero_state(n), n, gates)
    got, st = run(qs, n, 1, gates, fuse_k=5)
    assert st["tpb_gates"] > 0 and st["tc_blocks"] > 0
    assert np.max(np.abs(got - want)) <= TOL_C64
    assert fidelity_gap(got, want) <= 1e-6


def test_hadamard_layer_30q(qs):
    """The paper's 30-qubit Hadamard benchmark on a 16 GiB complex128 state: every amplitude
    2^-15 (sampled), the norm 1."""
    n = 30
    h = qs.qs_create(n, 2)
    try:
        qs.qs_apply_circuit(h, [("h", (q,), ()) for q in range(n)])
        st = qs.qs_last_stats(h)
        assert st["tpb_gates"] == n and st["passes"] == 1
        for off in (0, 12345678, (1 << n) - 4096):
            a = qs.qs_amplitudes(h, off, 4096)
            assert np.max(np.abs(a - 2.0 ** -15)) <= 1e-16
        assert abs(qs.qs_norm(h) - 1.0) <= 1e-12
    finally:
        qs.qs_destroy(h)
