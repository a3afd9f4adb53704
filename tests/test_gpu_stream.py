"""GPU parity of the streaming path (one kernel launch per gate) and the reductions,
through the C ABI, against the FP64 CPU oracle on identical seeded inputs."""
import math

import numpy as np
import pytest

import oracle
from paper_2409_14697_gb300 import inputs
from tests.gpu_util import TOL_C128, TOL_C64, fidelity_gap, require_gpu

pytestmark = pytest.mark.gpu

ALL_1Q = ["h", "x", "y", "z", "s", "t", "rx", "ry", "rz", "p", "u3"]
ALL_2Q = ["cnot", "cz", "swap", "cu3", "cp", "rzz"]


@pytest.fixture(scope="module")
def qs():
    require_gpu()
    from paper_2409_14697_gb300 import qs as q
    q.load()
    return q


def run_gpu(qs, n, dtype, psi0, gates, mode, **kw):
    h = qs.qs_create(n, dtype)
    try:
        qs.qs_set_amplitudes(h, psi0)
        qs.qs_apply_circuit(h, gates, qs.options(mode=mode, **kw))
        return qs.qs_amplitudes(h).astype(np.complex128)
    finally:
        qs.qs_destroy(h)


def check(got, want, dtype):
    err = np.max(np.abs(got - want))
    if dtype == 2:
        assert err <= TOL_C128, err
    else:
        assert err <= TOL_C64, err


@pytest.mark.parametrize("dtype", [2, 1])
@pytest.mark.parametrize("n", [1, 2, 3, 5, 8])
def test_every_gate_every_target(qs, n, dtype):
    psi0 = inputs.gaussian_state(n, seed=n)
    if dtype == 1:
        psi0 = psi0.astype(np.complex64)
    r = np.random.default_rng(n)
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
    # one gate per call, each compared with the oracle
    h = qs.qs_create(n, dtype)
    try:
        qs.qs_set_amplitudes(h, psi0)
        want = psi0.astype(np.complex128)
        for g in gates:
            qs.qs_apply_circuit(h, [g], qs.options(mode=qs.QS_MODE_GATE))
            oracle.run(want, n, [g])
            got = qs.qs_amplitudes(h).astype(np.complex128)
            err = np.max(np.abs(got - want))
            assert err <= (TOL_C128 if dtype == 2 else TOL_C64), (g, err)
            if dtype == 1:   # keep the comparison per gate: restart from the GPU state
                want = got.copy()
    finally:
        qs.qs_destroy(h)


@pytest.mark.parametrize("dtype", [2, 1])
@pytest.mark.parametrize("n", [3, 12])
def test_gate_mode_folded_rz_phases(qs, n, dtype):
    """Many RZ in one gate-by-gate call, mixed with H, CNOT and P: every RZ but the last
    runs as diag(1, e^{i theta}) on the half of the state with the target bit set and the
    collected global phase rides on the last one, so the state after the call equals the
    oracle's element by element, and the call's byte count shows the half passes."""
    psi0 = inputs.gaussian_state(n, seed=40 + n)
    if dtype == 1:
        psi0 = psi0.astype(np.complex64)
    r = np.random.default_rng(41 + n)
    gates = []
    for i in range(3 * n):
        q = i % n
        gates.append(("rz", (q,), (float(r.uniform(0, 2 * math.pi)),)))
        if i % 4 == 1:
            gates.append(("h", ((q + 1) % n,), ()))
        if i % 5 == 2:
            gates.append(("cnot", (q, (q + 2) % n), ()))
        if i % 7 == 3:
            gates.append(("p", (q,), (float(r.uniform(0, 2 * math.pi)),)))
    gates.append(("u3", (0,), tuple(float(a) for a in r.uniform(0, 2 * math.pi, 3))))
    h = qs.qs_create(n, dtype)
    try:
        qs.qs_set_amplitudes(h, psi0)
        qs.qs_apply_circuit(h, gates, qs.options(mode=qs.QS_MODE_GATE))
        st = qs.qs_last_stats(h)
        got = qs.qs_amplitudes(h).astype(np.complex128)
    finally:
        qs.qs_destroy(h)
    want = psi0.astype(np.complex128)
    oracle.run(want, n, gates)
    check(got, want, dtype)
    # bytes: read + write of the changed amplitudes, whole 32-byte sectors
    B = 16 if dtype == 2 else 8
    sb = 1 if dtype == 2 else 2
    full = 2.0 * B * (1 << n)
    last_rz = max(i for i, g in enumerate(gates) if g[0] == "rz")
    want_bytes = 0.0
    for i, (name, qb, _) in enumerate(gates):
        if name in ("rz", "p"):
            half = qb[0] >= sb and (name == "p" or i != last_rz)
            want_bytes += full / 2 if half else full
        elif name == "cnot":
            want_bytes += full / 2 if qb[0] >= sb else full
        else:
            want_bytes += full
    assert st["bytes"] == pytest.approx(want_bytes, rel=1e-12)


@pytest.mark.parametrize("dtype", [2, 1])
@pytest.mark.parametrize("n", [4, 12])
def test_gate_mode_deferred_hadamard_scale(qs, n, dtype):
    """Over 200 Hadamards in one gate-by-gate call, mixed with U3, CNOT and RZ: complex128
    runs all but every 64th and the last as the unscaled butterfly and lets the next scaled
    one carry 2^(-k/2); the state after the call equals the oracle's element by element."""
    psi0 = inputs.gaussian_state(n, seed=50 + n)
    if dtype == 1:
        psi0 = psi0.astype(np.complex64)
    r = np.random.default_rng(51 + n)
    gates = []
    for i in range(210):
        q = int(r.integers(n))
        gates.append(("h", (q,), ()))
        if i % 9 == 4:
            gates.append(("u3", ((q + 1) % n,), tuple(float(a) for a in r.uniform(0, 2 * math.pi, 3))))
        if i % 11 == 5:
            gates.append(("cnot", (q, (q + 1) % n), ()))
        if i % 13 == 6:
            gates.append(("rz", (q,), (float(r.uniform(0, 2 * math.pi)),)))
    gates.append(("x", (0,), ()))
    got = run_gpu(qs, n, dtype, psi0, gates, qs.QS_MODE_GATE)
    want = psi0.astype(np.complex128)
    oracle.run(want, n, gates)
    check(got, want, dtype)


@pytest.mark.parametrize("dtype", [2, 1])
def test_pinned_host_copies(qs, dtype):
    """Page-locked host buffers of 4 MiB or more take the copy-kernel path in both
    directions (whole state and an odd sub-range); every byte must round-trip, and the
    pageable path must give the same bytes."""
    torch = pytest.importorskip("torch")
    n = 20 if dtype == 2 else 21
    npdt = np.complex128 if dtype == 2 else np.complex64
    psi = inputs.gaussian_state(n, seed=77).astype(npdt)
    pin_in = torch.empty(psi.view(np.uint8).size, dtype=torch.uint8, pin_memory=True)
    assert pin_in.is_pinned()
    pin_in.numpy()[:] = psi.view(np.uint8)
    pin_out = torch.zeros_like(pin_in).pin_memory()
    h = qs.qs_create(n, dtype)
    try:
        qs.qs_set_amplitudes_from(h, 0, 1 << n, pin_in.data_ptr())
        assert np.array_equal(qs.qs_amplitudes(h), psi)           # pageable read-back
        qs.qs_amplitudes_into(h, 0, 1 << n, pin_out.data_ptr())
        assert np.array_equal(pin_out.numpy().view(npdt), psi)
        # odd offset and count (8-byte aligned for complex64): 3/4 of the state
        off, cnt = 3, (3 << (n - 2)) + 1
        B = psi.itemsize
        scaled = (psi * npdt(0.5)).astype(npdt)
        src = torch.empty(scaled.view(np.uint8).size, dtype=torch.uint8, pin_memory=True)
        src.numpy()[:] = scaled.view(np.uint8)
        qs.qs_set_amplitudes_from(h, off, cnt, src.data_ptr() + off * B)
        want = psi.copy()
        want[off:off + cnt] = scaled[off:off + cnt]
        assert np.array_equal(qs.qs_amplitudes(h), want)
        pin_out.zero_()
        qs.qs_amplitudes_into(h, off, cnt, pin_out.data_ptr() + off * B)
        got = pin_out.numpy().view(npdt)
        assert np.array_equal(got[off:off + cnt], want[off:off + cnt])
        assert not got[:off].any() and not got[off + cnt:].any()
    finally:
        qs.qs_destroy(h)


def test_async_copies_two_states(qs):
    """Stream-ordered copies on two states in flight (as the end-to-end benchmark runs them):
    pinned input shared by both, a circuit per state, each state's result into its own
    pinned buffer; after qs_synchronize both equal the oracle."""
    torch = pytest.importorskip("torch")
    n = 19
    psi = inputs.gaussian_state(n, seed=91)
    pin_in = torch.empty(psi.view(np.float64).size, dtype=torch.float64, pin_memory=True)
    pin_in.numpy()[:] = psi.view(np.float64)
    outs = [torch.zeros_like(pin_in).pin_memory() for _ in range(2)]
    circuits = [inputs.gate_sweep(n, "u3", seed=5, count=n) + inputs.gate_sweep(n, "cnot", seed=5, count=n),
                inputs.gate_sweep(n, "h", seed=6, count=n) + inputs.gate_sweep(n, "rz", seed=6, count=n)]
    hs = [qs.qs_create(n, 2) for _ in range(2)]
    try:
        for h, circ, out in zip(hs, circuits, outs):
            qs.qs_set_amplitudes_async(h, 0, 1 << n, pin_in.data_ptr())
            qs.qs_apply_circuit(h, circ, qs.options(mode=qs.QS_MODE_GATE))
            qs.qs_amplitudes_async(h, 0, 1 << n, out.data_ptr())
        for h in hs:
            qs.qs_synchronize(h)
    finally:
        for h in hs:
            qs.qs_destroy(h)
    for circ, out in zip(circuits, outs):
        want = psi.copy()
        oracle.run(want, n, circ)
        check(out.numpy().view(np.complex128), want, 2)


@pytest.mark.parametrize("dtype", [2, 1])
def test_async_copies_pageable_and_small(qs, dtype):
    """Stream-ordered copies from and to pageable numpy memory, and below the 4 MiB kernel
    threshold: the same bytes as the synchronous copies."""
    n = 12
    npdt = np.complex128 if dtype == 2 else np.complex64
    psi = inputs.gaussian_state(n, seed=93).astype(npdt)
    out = np.zeros_like(psi)
    h = qs.qs_create(n, dtype)
    try:
        qs.qs_set_amplitudes_async(h, 0, 1 << n, psi.ctypes.data)
        qs.qs_synchronize(h)
        assert np.array_equal(qs.qs_amplitudes(h), psi)
        qs.qs_amplitudes_async(h, 5, 100, out.ctypes.data + 5 * psi.itemsize)
        qs.qs_synchronize(h)
        assert np.array_equal(out[5:105], psi[5:105])
        assert not out[:5].any() and not out[105:].any()
    finally:
        qs.qs_destroy(h)


@pytest.mark.parametrize("dtype", [2, 1])
def test_brickwork_12q(qs, dtype):
    """20 layers of U3 on every qubit + CZ brickwork from |0...0>, all 4096 amplitudes."""
    n = 12
    gates = inputs.brickwork(n, 20, seed=1)
    want = oracle.run(oracle.zero_state(n), n, gates)
    psi0 = oracle.zero_state(n).astype(np.complex64 if dtype == 1 else np.complex128)
    got = run_gpu(qs, n, dtype, psi0, gates, qs.QS_MODE_GATE)
    check(got, want, dtype)
    if dtype == 1:
        assert fidelity_gap(got, want) < 1e-6


@pytest.mark.parametrize("k", [1, 2, 3, 4, 5, 6])
@pytest.mark.parametrize("dtype", [2, 1])
def test_dense_blocks(qs, k, dtype):
    n = 10
    r = np.random.default_rng(k)
    gates = []
    for i in range(6):
        qubits = tuple(int(x) for x in r.choice(n, size=k, replace=False))
        gates.append(("dense", qubits, inputs.random_unitary(k, seed=10 * k + i)))
    psi0 = inputs.gaussian_state(n, seed=3)
    want = oracle.run(psi0.copy(), n, gates)
    if dtype == 1:
        psi0 = psi0.astype(np.complex64)
    got = run_gpu(qs, n, dtype, psi0, gates, qs.QS_MODE_GATE)
    check(got, want, dtype)


@pytest.mark.parametrize("dtype", [2, 1])
@pytest.mark.parametrize("fk", [2, 3, 4, 5])
def test_fused_mode(qs, dtype, fk):
    n = 11
    gates = inputs.random_circuit(n, 120, seed=fk) + inputs.brickwork(n, 4, seed=fk)
    psi0 = inputs.gaussian_state(n, seed=fk)
    want = oracle.run(psi0.copy(), n, gates)
    if dtype == 1:
        psi0 = psi0.astype(np.complex64)
    got = run_gpu(qs, n, dtype, psi0, gates, qs.QS_MODE_FUSED, fuse_k=fk)
    check(got, want, dtype)


@pytest.mark.parametrize("dtype", [2, 1])
@pytest.mark.parametrize("n", [1, 3, 9, 13, 16, 21, 24])
def test_norm_expz(qs, n, dtype):
    psi = inputs.gaussian_state(n, seed=100 + n)
    psi = psi * 1.7  # not normalised on purpose
    if dtype == 1:
        psi = psi.astype(np.complex64)
    ref = psi.astype(np.complex128)
    h = qs.qs_create(n, dtype)
    try:
        qs.qs_set_amplitudes(h, psi)
        ez, nrm = qs.qs_expectation_z(h)
        nrm2 = qs.qs_norm(h)
    finally:
        qs.qs_destroy(h)
    want_n = oracle.norm(ref, n)
    want_z = oracle.expz(ref, n)
    assert abs(nrm - want_n) <= 1e-13 * want_n
    assert nrm2 == nrm
    assert np.max(np.abs(ez - want_z)) <= 1e-13 * want_n


@pytest.mark.parametrize("dtype", [2, 1])
@pytest.mark.parametrize("n,k", [(4, 16), (10, 1), (10, 37), (14, 1024), (18, 1024), (20, 4096)])
def test_top_k(qs, n, k, dtype):
    psi = inputs.gaussian_state(n, seed=200 + n)
    if dtype == 1:
        psi = psi.astype(np.complex64)
    ref = psi.astype(np.complex128)
    h = qs.qs_create(n, dtype)
    try:
        qs.qs_set_amplitudes(h, psi)
        idx, amp = qs.qs_top_amplitudes(h, k)
    finally:
        qs.qs_destroy(h)
    widx, wamp = oracle.top_k(ref, n, k)
    # probabilities are computed in FP64 on both sides from identical stored values,
    # so the selection and the tie order are identical
    assert np.array_equal(idx, widx)
    assert np.array_equal(amp, wamp)


def test_top_k_ties_uniform(qs):
    n = 12
    h = qs.qs_create(n, 2)
    try:
        qs.qs_apply_circuit(h, [("h", (q,), ()) for q in range(n)], qs.options(mode=qs.QS_MODE_GATE))
        idx, amp = qs.qs_top_amplitudes(h, 100)
    finally:
        qs.qs_destroy(h)
    assert list(idx) == list(range(100))   # all equal: lowest indices first


@pytest.mark.parametrize("n,k", [(14, 100), (15, 4096)])
def test_top_k_ties_uniform_beyond_candidate_cap(qs, n, k):
    """2^n equal probabilities (more than the fast path's 8192 candidates): the exact radix
    pipeline runs and the lowest indices come first."""
    h = qs.qs_create(n, 2)
    try:
        qs.qs_apply_circuit(h, [("h", (q,), ()) for q in range(n)], qs.options(mode=qs.QS_MODE_GATE))
        idx, amp = qs.qs_top_amplitudes(h, k)
    finally:
        qs.qs_destroy(h)
    assert list(idx) == list(range(k))


@pytest.mark.parametrize("dtype", [2, 1])
@pytest.mark.parametrize("n,k,levels", [(16, 1024, 5), (18, 333, 40), (20, 4096, 3)])
def test_top_k_discrete_magnitudes(qs, n, k, levels, dtype):
    """Probabilities from a few exact values (heavy ties at and around the K-th one)."""
    r = np.random.default_rng(n + levels)
    mags = r.uniform(0.1, 1.0, size=levels)[r.integers(levels, size=1 << n)]
    psi = mags * np.array([1, 1j, -1, -1j])[r.integers(4, size=1 << n)]  # exact phases: exact ties
    psi = psi.astype(np.complex64 if dtype == 1 else np.complex128)
    ref = psi.astype(np.complex128)
    h = qs.qs_create(n, dtype)
    try:
        qs.qs_set_amplitudes(h, psi)
        idx, amp = qs.qs_top_amplitudes(h, k)
    finally:
        qs.qs_destroy(h)
    widx, wamp = oracle.top_k(ref, n, k)
    assert np.array_equal(idx, widx)
    assert np.array_equal(amp, wamp)


def test_top_k_sparse_state_zero_threshold(qs):
    """Fewer nonzero amplitudes than K: the K-th probability is 0 (ties among zeros go to
    the lowest indices)."""
    n, k = 15, 2000
    r = np.random.default_rng(4)
    psi = np.zeros(1 << n, dtype=np.complex128)
    nz = r.choice(1 << n, size=500, replace=False)
    psi[nz] = r.standard_normal(500) + 1j * r.standard_normal(500)
    h = qs.qs_create(n, 2)
    try:
        qs.qs_set_amplitudes(h, psi)
        idx, amp = qs.qs_top_amplitudes(h, k)
    finally:
        qs.qs_destroy(h)
    widx, wamp = oracle.top_k(psi, n, k)
    assert np.array_equal(idx, widx)
    assert np.array_equal(amp, wamp)


def test_invalid_records(qs):
    h = qs.qs_create(4, 2)
    try:
        for bad in [[("cnot", (1, 1), ())], [("h", (4,), ())], [("h", (-1,), ())]]:
            with pytest.raises(qs.QsError) as e:
                qs.qs_apply_circuit(h, bad)
            assert e.value.code == qs.QS_ERR_INVALID
        with pytest.raises(qs.QsError):
            qs.qs_amplitudes(h, 10, 10)
    finally:
        qs.qs_destroy(h)


def test_reset_and_renormalize(qs):
    n = 9
    h = qs.qs_create(n, 2)
    try:
        psi = inputs.gaussian_state(n, seed=5) * 3.0
        qs.qs_set_amplitudes(h, psi)
        old = qs.qs_renormalize(h)
        assert abs(old - 9.0) < 1e-12
        assert abs(qs.qs_norm(h) - 1.0) < 1e-14
        qs.qs_reset(h)
        got = qs.qs_amplitudes(h)
        assert got[0] == 1 and np.count_nonzero(got) == 1
    finally:
        qs.qs_destroy(h)
