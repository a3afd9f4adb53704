"""GPU parity of the planned in-cache path (chunk kernel, TMA-staged tiles) against
the FP64 oracle, and kernel-selection equivalence at sizes beyond the oracle's reach."""
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


def run_gpu(qs, n, dtype, psi0, gates, mode, **kw):
    h = qs.qs_create(n, dtype)
    try:
        if psi0 is not None:
            qs.qs_set_amplitudes(h, psi0)
        qs.qs_apply_circuit(h, gates, qs.options(mode=mode, **kw))
        stats = qs.qs_last_stats(h)
        return qs.qs_amplitudes(h).astype(np.complex128), stats
    finally:
        qs.qs_destroy(h)


def tol(dtype):
    return TOL_C128 if dtype == 2 else TOL_C64


@pytest.mark.parametrize("dtype", [2, 1])
@pytest.mark.parametrize("n,m", [(5, 0), (8, 6), (12, 0), (14, 8), (16, 10), (17, 0), (20, 12)])
def test_random_circuits_chunked(qs, n, m, dtype):
    gates = inputs.random_circuit(n, 200, seed=n + m) + inputs.brickwork(n, 6, seed=n)
    psi0 = inputs.gaussian_state(n, seed=n)
    want = oracle.run(psi0.copy(), n, gates)
    if dtype == 1:
        psi0 = psi0.astype(np.complex64)
    got, st = run_gpu(qs, n, dtype, psi0, gates, qs.QS_MODE_AUTO, chunk_m=m)
    assert np.max(np.abs(got - want)) <= tol(dtype)
    assert st["passes"] <= len(gates)


@pytest.mark.parametrize("dtype", [2, 1])
@pytest.mark.parametrize("fk", [1, 2, 3, 4])
def test_fusion_inside_passes(qs, dtype, fk):
    n = 16
    gates = inputs.brickwork(n, 8, seed=5) + inputs.random_circuit(n, 60, seed=fk)
    psi0 = inputs.gaussian_state(n, seed=6)
    want = oracle.run(psi0.copy(), n, gates)
    if dtype == 1:
        psi0 = psi0.astype(np.complex64)
    got, _ = run_gpu(qs, n, dtype, psi0, gates, qs.QS_MODE_AUTO, fuse_k=fk, chunk_m=9)
    assert np.max(np.abs(got - want)) <= tol(dtype)


@pytest.mark.parametrize("dtype", [2, 1])
def test_dense_user_blocks_in_passes(qs, dtype):
    n = 15
    gates = []
    for i, k in enumerate([1, 2, 3, 4, 5, 6, 3, 4]):
        r = np.random.default_rng(i)
        qubits = tuple(int(x) for x in r.choice(n, size=k, replace=False))
        gates.append(("dense", qubits, inputs.random_unitary(k, seed=i)))
        gates += inputs.random_circuit(n, 10, seed=100 + i)
    psi0 = inputs.gaussian_state(n, seed=8)
    want = oracle.run(psi0.copy(), n, gates)
    if dtype == 1:
        psi0 = psi0.astype(np.complex64)
    got, _ = run_gpu(qs, n, dtype, psi0, gates, qs.QS_MODE_AUTO, chunk_m=10)
    assert np.max(np.abs(got - want)) <= tol(dtype)


@pytest.mark.parametrize("dtype", [2, 1])
@pytest.mark.parametrize("family", ["qaoa", "tfim", "qft", "ghz"])
def test_circuit_families(qs, dtype, family):
    n = 18
    if family == "qaoa":
        gates = inputs.qaoa_3regular(n, p=4, seed=1)
    elif family == "tfim":
        gates = inputs.tfim(n, steps=20, dt=0.05)
    elif family == "qft":
        gates = inputs.qft(n)
    else:
        gates = [("h", (0,), ())] + [("cnot", (q, q + 1), ()) for q in range(n - 1)]
    want = oracle.run(oracle.zero_state(n), n, gates)
    psi0 = oracle.zero_state(n).astype(np.complex64 if dtype == 1 else np.complex128)
    got, st = run_gpu(qs, n, dtype, psi0, gates, qs.QS_MODE_AUTO)
    assert np.max(np.abs(got - want)) <= tol(dtype)
    if dtype == 1:
        assert fidelity_gap(got, want) <= 1e-6


@pytest.mark.parametrize("dtype", [2, 1])
def test_config1_brickwork_12q_auto(qs, dtype):
    """The 12-qubit workload.  complex64: one tile holds the whole state, one pass for 350
    gates.  complex128 (FP64-bound): tiles of 2^7 amplitudes, so 32 SMs share the work in
    several passes; the same result either way, and with the one-tile plan."""
    n = 12
    gates = inputs.brickwork(n, 20, seed=1)
    want = oracle.run(oracle.zero_state(n), n, gates)
    psi0 = oracle.zero_state(n).astype(np.complex64 if dtype == 1 else np.complex128)
    got, st = run_gpu(qs, n, dtype, psi0, gates, qs.QS_MODE_AUTO)
    assert np.max(np.abs(got - want)) <= tol(dtype)
    if dtype == 1:
        assert st["passes"] == 1
    else:
        assert 1 < st["passes"] < len(gates) / 4
        got1, st1 = run_gpu(qs, n, dtype, psi0, gates, qs.QS_MODE_AUTO, chunk_m=12)
        assert np.max(np.abs(got1 - want)) <= tol(dtype)
        assert st1["passes"] == 1


@pytest.mark.parametrize("dtype", [2, 1])
def test_mode_equivalence_24q(qs, dtype):
    """GATE, AUTO and FUSED agree at 24 qubits on a brickwork + sweep circuit."""
    n = 24
    gates = inputs.brickwork(n, 6, seed=2) + inputs.sweep_all(n, seed=3, count=n)
    psi0 = inputs.gaussian_state(n, seed=9)
    if dtype == 1:
        psi0 = psi0.astype(np.complex64)
    a, _ = run_gpu(qs, n, dtype, psi0, gates, qs.QS_MODE_GATE)
    b, sb = run_gpu(qs, n, dtype, psi0, gates, qs.QS_MODE_AUTO)
    c, _ = run_gpu(qs, n, dtype, psi0, gates, qs.QS_MODE_FUSED, fuse_k=3)
    t = 1e-12 if dtype == 2 else 2e-5
    assert np.max(np.abs(a - b)) <= t
    assert np.max(np.abs(a - c)) <= t
    assert sb["passes"] < len(gates) / 3


def test_inverse_returns_initial_26q(qs):
    """circuit followed by its inverse returns the initial state (complex128, 26 qubits)."""
    n = 26
    gates = inputs.brickwork(n, 8, seed=4) + inputs.sweep_all(n, seed=4, count=n)
    full = gates + inputs.inverse(gates)
    psi0 = inputs.gaussian_state(n, seed=10)
    got, _ = run_gpu(qs, n, 2, psi0, full, qs.QS_MODE_AUTO)
    assert np.max(np.abs(got - psi0)) <= 1e-12


def _run_c64(qs, n, psi0, gates, phases=True, **kw):
    h = qs.qs_create(n, 1)
    try:
        qs.qs_set_amplitudes(h, psi0)
        o = qs.options(**kw)
        if not phases:
            o.flags |= qs.QS_OPT_NO_REG_PHASES
        qs.qs_apply_circuit(h, gates, o)
        return qs.qs_amplitudes(h).astype(np.complex128), qs.qs_last_stats(h)
    finally:
        qs.qs_destroy(h)


@pytest.mark.parametrize("n", [13, 14, 17])
@pytest.mark.parametrize("fk", [1, 2])
def test_register_phases_match_plain_sweeps(qs, n, fk):
    """complex64 passes over 2^13-amplitude tiles with register phases (default) against
    the same passes with one shared-memory sweep per op, and both against the oracle.  The
    circuit mixes every gate type a phase holds (one-qubit dense, H, X, diagonals,
    controlled gates with the control inside and outside the register positions, CZ, CP,
    RZZ) with the ones it leaves to plain sweeps (SWAP, dense two-qubit blocks)."""
    gates = inputs.brickwork(n, 10, seed=fk) + inputs.random_circuit(n, 300, seed=40 + fk + n) + \
        inputs.qaoa_3regular(n, p=1, seed=fk) + inputs.qft(n)
    gates.append(("dense", (3, n - 1), inputs.random_unitary(2, seed=fk)))
    gates += inputs.random_circuit(n, 40, seed=7 + n)
    psi0 = inputs.gaussian_state(n, seed=fk + n).astype(np.complex64)
    want = oracle.run(psi0.astype(np.complex128), n, gates)
    a, sa = _run_c64(qs, n, psi0, gates, True, fuse_k=fk)
    b, sb = _run_c64(qs, n, psi0, gates, False, fuse_k=fk)
    assert np.max(np.abs(a - want)) <= TOL_C64
    assert np.max(np.abs(b - want)) <= TOL_C64
    assert fidelity_gap(a, want) <= 1e-6
    # register phases take several ops per shared-memory sweep
    assert sa["tile_sweeps"] <= sb["tile_sweeps"]
    if fk == 1:
        assert 2 * sa["tile_sweeps"] < sb["tile_sweeps"]


def test_register_phases_brickwork_sweeps(qs):
    """On brickwork, a phase holds many gates: far fewer tile sweeps than ops."""
    n = 20
    gates = inputs.brickwork(n, 12, seed=9)
    psi0 = oracle.zero_state(n).astype(np.complex64)
    want = oracle.run(oracle.zero_state(n), n, gates)
    a, st = _run_c64(qs, n, psi0, gates, True, fuse_k=1)
    assert np.max(np.abs(a - want)) <= TOL_C64
    assert st["tile_sweeps"] * 4 <= st["ops_after_fuse"]


def test_fusion_cost_counts_one_qubit_forms(qs):
    """complex128 fusion counts each one-qubit matrix at the FP64 cost of its form: RX, RY
    (4 per amplitude) and U3 (7) on different qubits stay apart, because a 4x4 block costs
    16 (U3 then split into a real rotation and phases: at least as many ops as gates); H
    then U3 on one qubit merge (8 against 3 + 7).  Parity with the oracle either way."""
    n = 14
    r = np.random.default_rng(3)
    layer = [("rx", (q,), (float(r.uniform(0, 6.28)),)) for q in range(n)]
    layer += [("ry", (q,), (float(r.uniform(0, 6.28)),)) for q in range(n)]
    layer += [("u3", (q,), tuple(float(x) for x in r.uniform(0, 6.28, 3))) for q in range(n)]
    psi0 = inputs.gaussian_state(n, seed=3)
    want = oracle.run(psi0.copy(), n, layer)
    got, st = run_gpu(qs, n, 2, psi0, layer, qs.QS_MODE_AUTO, chunk_m=8, fuse_k=2)
    assert np.max(np.abs(got - want)) <= TOL_C128
    assert st["ops_after_fuse"] >= len(layer)
    pairs = []
    for q in range(n):
        pairs += [("h", (q,), ()), ("u3", (q,), tuple(float(x) for x in r.uniform(0, 6.28, 3)))]
    want = oracle.run(psi0.copy(), n, pairs)
    got, st = run_gpu(qs, n, 2, psi0, pairs, qs.QS_MODE_AUTO, chunk_m=8, fuse_k=2)
    assert np.max(np.abs(got - want)) <= TOL_C128
    assert st["ops_after_fuse"] == n


def _nonlocal_phase_circuit(n, seed):
    """QFT, then a seeded mix of H, U3, CNOT, RZ and controlled phases (CP, CZ and CU3 with
    theta = 0, a phase on the target chosen by the control)."""
    r = np.random.default_rng(seed)
    gates = list(inputs.qft(n))
    for _ in range(300):
        a, b = (int(x) for x in r.choice(n, 2, replace=False))
        kind = int(r.integers(7))
        if kind == 0:
            gates.append(("h", (a,), ()))
        elif kind == 1:
            gates.append(("u3", (a,), tuple(float(x) for x in r.uniform(0, 2 * np.pi, 3))))
        elif kind == 2:
            gates.append(("cnot", (a, b), ()))
        elif kind == 3:
            gates.append(("rz", (a,), (float(r.uniform(0, 2 * np.pi)),)))
        elif kind == 4:
            gates.append(("cp", (a, b), (float(r.uniform(0, 2 * np.pi)),)))
        elif kind == 5:
            gates.append(("cz", (a, b), ()))
        else:
            gates.append(("cu3", (a, b), (0.0, float(r.uniform(0, 2 * np.pi)), float(r.uniform(0, 2 * np.pi)))))
    return gates


@pytest.mark.parametrize("prec", [1, 2])
@pytest.mark.parametrize("n,m", [(14, 6), (18, 8), (20, 12)])
@pytest.mark.parametrize("mode", ["auto", "chunk"])
def test_nonlocal_controlled_phases(qs, n, m, prec, mode):
    """complex128 passes take controlled phases whose other qubit is outside the local set
    (a per-tile factor folded into the block's table).  The plan must use that (some
    controlled phase in a pass with one of its qubits non-local), and the state must equal
    the oracle's with FP64 and with double-float arithmetic."""
    gates = _nonlocal_phase_circuit(n, seed=n + m)
    pog, lm = qs.qs_plan(n, 2, gates, qs.options(chunk_m=m))
    hi = 0
    for (name, qb, _), p in zip(gates, pog):
        L = int(lm[p])
        if L and name in ("cp", "cz", "cu3") and len(qb) == 2:
            if sum((L >> q) & 1 for q in qb) == 1:
                hi += 1
    assert hi > 0
    psi0 = inputs.gaussian_state(n, seed=n + 1)
    want = oracle.run(psi0.copy(), n, gates)
    md = qs.QS_MODE_AUTO if mode == "auto" else qs.QS_MODE_CHUNK   # chunk: single-op passes too
    got, st = run_gpu(qs, n, 2, psi0, gates, md, chunk_m=m, precision=prec)
    assert np.max(np.abs(got - want)) <= TOL_C128
    if mode == "auto":
        assert st["passes"] == len(lm)


@pytest.mark.parametrize("dtype,flags", [(2, 0), (1, 1)])
@pytest.mark.parametrize("n", [14, 20])
def test_qft_merged_diagonal_blocks(qs, n, dtype, flags):
    """QFT: each target's run of controlled phases is merged into diagonal blocks of up
    to 8 qubits inside the tile passes (complex128, and complex64 without register phases);
    against the oracle and the inverse QFT."""
    gates = inputs.qft(n)
    psi0 = inputs.gaussian_state(n, seed=n)
    want = oracle.run(psi0.copy(), n, gates)
    p0 = psi0.astype(np.complex64 if dtype == 1 else np.complex128)
    got, st = run_gpu(qs, n, dtype, p0, gates, qs.QS_MODE_AUTO, **({"flags": flags} if flags else {}))
    assert np.max(np.abs(got - want)) <= tol(dtype)
    # fewer tile sweeps than ops: the controlled phases of a target share blocks
    assert st["tile_sweeps"] < len(gates)


@pytest.mark.parametrize("prec", [1, 2])
@pytest.mark.parametrize("n,m", [(14, 0), (18, 8), (20, 12)])
def test_qft_hadamard_joined_with_controlled_block(qs, n, m, prec):
    """complex128 FP64 passes apply an unscaled Hadamard and the next diagonal block
    controlled by its qubit (a QFT target's controlled phases, with factors from
    non-local partners where the tile is narrower than the state) in one sweep: fewer
    sweeps than ops after the merge (chunk mode: every pass a tile pass).  Double-float
    keeps them apart.  Oracle parity for both."""
    gates = inputs.qft(n)
    psi0 = inputs.gaussian_state(n, seed=3 * n + m)
    want = oracle.run(psi0.copy(), n, gates)
    got, st = run_gpu(qs, n, 2, psi0, gates, qs.QS_MODE_CHUNK, chunk_m=m, precision=prec)
    assert np.max(np.abs(got - want)) <= TOL_C128
    if prec == 1:
        assert st["tile_sweeps"] < st["ops_after_fuse"]
    else:
        assert st["tile_sweeps"] == st["ops_after_fuse"]


@pytest.mark.parametrize("n", [13, 20])
def test_register_phases_phase_layers(qs, n):
    """complex64 register phases with layers of one-qubit phases (S, T, P on every qubit),
    CZ brickwork and U3: runs of phases and sign pairs applied as one member, against the
    oracle."""
    r = np.random.default_rng(n)
    gates = []
    for layer in range(6):
        for q in range(n):
            name = ("s", "t", "p")[q % 3]
            gates.append((name, (q,), (float(r.uniform(0, 6.28)),) if name == "p" else ()))
        for a in range(layer % 2, n - 1, 2):
            gates.append(("cz", (a, a + 1), ()))
        for q in range(n):
            gates.append(("u3", (q,), tuple(float(x) for x in r.uniform(0, 6.28, 3))))
    psi0 = inputs.gaussian_state(n, seed=n).astype(np.complex64)
    want = oracle.run(psi0.astype(np.complex128), n, gates)
    got, st = _run_c64(qs, n, psi0, gates)
    assert np.max(np.abs(got - want)) <= TOL_C64
    assert fidelity_gap(got, want) <= 1e-6
