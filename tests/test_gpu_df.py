"""GPU parity of the complex128 double-float arithmetic mode (QS_PREC_DF32: FP64
storage, FP32-pair arithmetic with compensated products and sums) against the FP64
oracle, at the complex128 tolerance of 1e-12."""
import math

import numpy as np
import pytest

import oracle
from paper_2409_14697_gb300 import inputs
from tests.gpu_util import TOL_C128, require_gpu

pytestmark = pytest.mark.gpu

ALL_1Q = ["h", "x", "y", "z", "s", "t", "rx", "ry", "rz", "p", "u3"]
ALL_2Q = ["cnot", "cz", "swap", "cu3", "cp", "rzz"]


@pytest.fixture(scope="module")
def qs():
    require_gpu()
    from paper_2409_14697_gb300 import qs as q
    q.load()
    return q


def run(qs, n, psi0, gates, mode, prec):
    h = qs.qs_create(n, 2)
    try:
        qs.qs_set_amplitudes(h, psi0)
        qs.qs_apply_circuit(h, gates, qs.options(mode=mode, precision=prec))
        return qs.qs_amplitudes(h)
    finally:
        qs.qs_destroy(h)


@pytest.mark.parametrize("n", [1, 3, 8])
def test_every_gate_every_target_df(qs, n):
    r = np.random.default_rng(50 + n)
    gates = []
    for name in ALL_1Q:
        for q in range(n):
            gates.append((name, (q,), tuple(r.uniform(0, 2 * math.pi, inputs.n_params(name)))))
    if n >= 2:
        for name in ALL_2Q:
            for a in range(n):
                for b in range(n):
                    if a != b:
                        gates.append((name, (a, b), tuple(r.uniform(0, 2 * math.pi, inputs.n_params(name)))))
    gates += [("dense", (0,), inputs.random_unitary(1, seed=3))]
    if n >= 2:
        gates += [("dense", (n - 1, 0), inputs.random_unitary(2, seed=4))]
    psi0 = inputs.gaussian_state(n, seed=n)
    want = oracle.run(psi0.copy(), n, gates)
    got = run(qs, n, psi0, gates, qs.QS_MODE_GATE, qs.QS_PREC_DF32)
    assert np.max(np.abs(got - want)) <= TOL_C128


def test_brickwork_12q_df(qs):
    """350 gates from |0...0>: large amplitudes, exact zeros and ones at the start."""
    n = 12
    gates = inputs.brickwork(n, 20, seed=1)
    want = oracle.run(oracle.zero_state(n), n, gates)
    got = run(qs, n, oracle.zero_state(n), gates, qs.QS_MODE_GATE, qs.QS_PREC_DF32)
    err = np.max(np.abs(got - want))
    assert err <= TOL_C128
    assert err <= 1e-13      # double-float keeps ~2^-46 per update


def test_sweep_and_inverse_26q_df(qs):
    n = 26
    gates = inputs.sweep_all(n, seed=5, count=n)
    psi0 = inputs.gaussian_state(n, seed=11)
    got = run(qs, n, psi0, gates + inputs.inverse(gates), qs.QS_MODE_GATE, qs.QS_PREC_DF32)
    assert np.max(np.abs(got - psi0)) <= TOL_C128


def test_df_matches_fp64_24q(qs):
    n = 24
    gates = inputs.sweep_all(n, seed=6, count=n) + inputs.brickwork(n, 3, seed=6)
    psi0 = inputs.gaussian_state(n, seed=12) * 1.7   # unnormalised on purpose
    a = run(qs, n, psi0, gates, qs.QS_MODE_GATE, qs.QS_PREC_DF32)
    b = run(qs, n, psi0, gates, qs.QS_MODE_GATE, qs.QS_PREC_FP64)
    assert np.max(np.abs(a - b)) <= TOL_C128


def test_df_tiny_and_zero_amplitudes(qs):
    n = 6
    psi0 = np.zeros(1 << n, dtype=np.complex128)
    psi0[0] = 1.0
    psi0[5] = 1e-20 + 3e-30j
    psi0[9] = -2.5e-80
    gates = [("h", (q,), ()) for q in range(n)] + inputs.random_circuit(n, 40, seed=3)
    want = oracle.run(psi0.copy(), n, gates)
    got = run(qs, n, psi0, gates, qs.QS_MODE_GATE, qs.QS_PREC_DF32)
    assert np.max(np.abs(got - want)) <= TOL_C128


@pytest.mark.parametrize("n,m", [(12, 0), (16, 10), (20, 12)])
def test_planned_passes_df(qs, n, m):
    """Double-float arithmetic inside the in-cache chunk passes."""
    gates = inputs.brickwork(n, 10, seed=n) + inputs.random_circuit(n, 150, seed=m + 1)
    psi0 = inputs.gaussian_state(n, seed=n + 1)
    want = oracle.run(psi0.copy(), n, gates)
    h = qs.qs_create(n, 2)
    try:
        qs.qs_set_amplitudes(h, psi0)
        qs.qs_apply_circuit(h, gates, qs.options(chunk_m=m, precision=qs.QS_PREC_DF32))
        got = qs.qs_amplitudes(h)
    finally:
        qs.qs_destroy(h)
    assert np.max(np.abs(got - want)) <= TOL_C128


def test_planned_dense_blocks_df(qs):
    n = 14
    gates = []
    for i, k in enumerate([1, 2, 3, 4, 2, 3]):
        r = np.random.default_rng(i)
        qubits = tuple(int(x) for x in r.choice(n, size=k, replace=False))
        gates.append(("dense", qubits, inputs.random_unitary(k, seed=20 + i)))
        gates += inputs.random_circuit(n, 20, seed=30 + i)
    psi0 = inputs.gaussian_state(n, seed=2)
    want = oracle.run(psi0.copy(), n, gates)
    h = qs.qs_create(n, 2)
    try:
        qs.qs_set_amplitudes(h, psi0)
        qs.qs_apply_circuit(h, gates, qs.options(chunk_m=10, fuse_k=3, precision=qs.QS_PREC_DF32))
        got = qs.qs_amplitudes(h)
    finally:
        qs.qs_destroy(h)
    assert np.max(np.abs(got - want)) <= TOL_C128


@pytest.mark.parametrize("n", [14, 18])
def test_planned_qft_df_tiles(qs, n):
    """QFT with double-float tiles: merged controlled-phase blocks (F_CDIAGK) and H on
    float pairs held for the whole pass."""
    gates = inputs.qft(n)
    psi0 = inputs.gaussian_state(n, seed=n + 5)
    want = oracle.run(psi0.copy(), n, gates)
    got = run(qs, n, psi0, gates, qs.QS_MODE_AUTO, qs.QS_PREC_DF32)
    assert np.max(np.abs(got - want)) <= TOL_C128


def test_planned_long_circuit_df_tiles(qs):
    """Hundreds of ops inside each pass on float pairs (errors add over the ops of a pass,
    each op within ~2^-46 of sum |m x|)."""
    n = 16
    gates = inputs.brickwork(n, 40, seed=3) + inputs.qaoa_3regular(n, p=3, seed=3) + \
        inputs.tfim(n, steps=20, dt=0.05) + inputs.random_circuit(n, 400, seed=9)
    psi0 = inputs.gaussian_state(n, seed=11)
    want = oracle.run(psi0.copy(), n, gates)
    got = run(qs, n, psi0, gates, qs.QS_MODE_AUTO, qs.QS_PREC_DF32)
    assert np.max(np.abs(got - want)) <= TOL_C128
