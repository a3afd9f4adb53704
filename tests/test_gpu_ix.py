"""GPU parity of the integer-product arithmetic of complex128 streaming updates
(QS_PREC_IX64: one-qubit dense and diagonal gates as dot products of exact 64-bit integer
significand products, one rounding per output), through the C ABI.

* Every gate type on every target of a 12-qubit state, gate by gate, against the oracle
  (max-abs <= 1e-12) and against the native FP64 kernels (the two differ by rounding
  only).
* The U3, CU3 and RZ sweeps of the gate benchmark at 20 qubits against the oracle.
* Planned calls (chunk passes with one-qubit dense and diagonal tile ops, phase functions)
  of QFT, fully connected QAOA, TFIM, brickwork and U3 sweeps at 16 qubits, against the
  oracle and the native FP64 plan.
* Bit for bit against the host build of the same arithmetic (tests/ix_check.cpp): caller
  matrices (U3-class, general unitary, real rotation, RX-class, diagonal) on a 16-qubit
  Gaussian state.  Groups a
  thread gives to the native FP64 form (the first IX_NATIVE_GROUPS of every 4 groups of
  256 consecutive pairs, the streaming kernel's assignment) match the native FP64 kernel
  instead.
"""
import subprocess

import numpy as np
import pytest

import oracle
from paper_2409_14697_gb300 import inputs
from tests.gpu_util import TOL_C128, require_gpu
from tests.ix_build import build_ix_check

pytestmark = pytest.mark.gpu

# groups per thread and native FP64 groups per thread of the complex128 two-element kernels
IX_GROUPS_PER_THREAD = 4
IX_NATIVE_GROUPS = 1


@pytest.fixture(scope="module")
def qs():
    require_gpu()
    from paper_2409_14697_gb300 import qs as q
    q.load()
    return q


def _run(qs, n, psi, gates, prec):
    h = qs.qs_create(n, qs.QS_C128)
    try:
        qs.qs_set_amplitudes(h, psi)
        qs.qs_apply_circuit(h, gates, qs.options(mode=qs.QS_MODE_GATE, precision=prec))
        return qs.qs_amplitudes(h)
    finally:
        qs.qs_destroy(h)


ONE_QUBIT = ("h", "x", "y", "z", "s", "t", "rx", "ry", "rz", "p", "u3")
TWO_QUBIT = ("cnot", "cz", "swap", "cu3", "cp", "rzz")


def test_every_gate_every_target_12q(qs):
    n = 12
    r = inputs.rng(41)
    psi = inputs.gaussian_state(n, seed=41)
    gates = []
    for name in ONE_QUBIT:
        for q in range(n):
            gates.append((name, (q,), tuple(r.uniform(0, 2 * np.pi, inputs.n_params(name)))))
    for name in TWO_QUBIT:
        for q in range(n):
            gates.append((name, (q, (q + 1 + int(r.integers(n - 1))) % n),
                          tuple(r.uniform(0, 2 * np.pi, inputs.n_params(name)))))
    for q in range(n):
        gates.append(("dense", (q,), inputs.random_unitary(1, seed=100 + q)))
    want = oracle.run(psi.copy(), n, gates)
    got = _run(qs, n, psi, gates, qs.QS_PREC_IX64)
    nat = _run(qs, n, psi, gates, qs.QS_PREC_FP64)
    assert np.max(np.abs(got - want)) <= TOL_C128
    assert np.max(np.abs(got - nat)) <= 1e-14 * np.max(np.abs(want))


@pytest.mark.parametrize("name", ["u3", "cu3", "rz"])
def test_benchmark_sweeps_20q(qs, name):
    n = 20
    psi = inputs.gaussian_state(n, seed=2024)
    seg = inputs.gate_sweep(n, name, seed=2, count=3 * n)
    want = oracle.run(psi.copy(), n, seg)
    got = _run(qs, n, psi, seg, qs.QS_PREC_IX64)
    assert np.max(np.abs(got - want)) <= TOL_C128


FAMILIES = {
    "qft": lambda n: inputs.qft(n),
    "qaoa_complete_p5": lambda n: inputs.qaoa_complete(n, p=5, seed=5),
    "tfim20": lambda n: inputs.tfim(n, steps=20, dt=0.05),
    "brickwork10": lambda n: inputs.brickwork(n, 10, seed=12),
    "u3_sweep": lambda n: inputs.gate_sweep(n, "u3", seed=2, count=2 * n),
}


@pytest.mark.parametrize("family", list(FAMILIES))
@pytest.mark.parametrize("chunk_m", [0, 9])
def test_planned_circuits_vs_oracle(qs, family, chunk_m):
    """Planned calls (chunk passes, phase functions, streaming ops) with integer products:
    against the oracle and against the same plan in native FP64."""
    n = 16
    psi = inputs.gaussian_state(n, seed=61)
    gates = FAMILIES[family](n)
    want = oracle.run(psi.copy(), n, gates)
    h = qs.qs_create(n, qs.QS_C128)
    try:
        out = {}
        for prec in (qs.QS_PREC_IX64, qs.QS_PREC_FP64):
            qs.qs_set_amplitudes(h, psi)
            qs.qs_apply_circuit(h, gates, qs.options(chunk_m=chunk_m, precision=prec))
            out[prec] = qs.qs_amplitudes(h)
    finally:
        qs.qs_destroy(h)
    assert np.max(np.abs(out[qs.QS_PREC_IX64] - want)) <= TOL_C128
    assert np.max(np.abs(out[qs.QS_PREC_IX64] - out[qs.QS_PREC_FP64])) <= 1e-14 * np.max(np.abs(want))


@pytest.fixture(scope="module")
def ix_check(tmp_path_factory):
    return build_ix_check(tmp_path_factory.mktemp("ix_gpu"))


def _u3_class(seed):
    # a unitary with a real first entry (the 14-term form)
    u = inputs.random_unitary(1, seed=seed)
    u = u * np.exp(-1j * np.angle(u[0, 0]))
    u[0, 0] = abs(u[0, 0])    # exactly real (the product leaves a rounding residue)
    return u


@pytest.mark.parametrize("kind", ["r0", "gen", "real", "rx", "diag"])
@pytest.mark.parametrize("q", [0, 7, 15])
def test_bitwise_against_host_arithmetic(qs, ix_check, tmp_path, kind, q):
    n = 16
    psi = inputs.gaussian_state(n, seed=500 + q)
    if kind == "r0":
        u = _u3_class(700 + q)
    elif kind == "gen":
        u = inputs.random_unitary(1, seed=800 + q)
        assert u[0, 0].imag != 0
    elif kind == "real":
        a = inputs.rng(950 + q).uniform(0, 2 * np.pi)
        u = np.array([[np.cos(a), -np.sin(a)], [np.sin(a), np.cos(a)]], dtype=np.complex128)
    elif kind == "rx":
        a = inputs.rng(970 + q).uniform(0, 2 * np.pi)
        u = np.array([[np.cos(a), -1j * np.sin(a)], [-1j * np.sin(a), np.cos(a)]])
    else:
        a, b = inputs.rng(900 + q).uniform(0, 2 * np.pi, 2)
        u = np.diag([np.exp(1j * a), np.exp(1j * b)])
    gate = [("dense", (q,), u)]
    got = _run(qs, n, psi, gate, qs.QS_PREC_IX64)
    nat = _run(qs, n, psi, gate, qs.QS_PREC_FP64)
    (tmp_path / "psi.bin").write_bytes(np.ascontiguousarray(psi).tobytes())
    (tmp_path / "m.bin").write_bytes(np.ascontiguousarray(u, dtype=np.complex128).reshape(-1).view(np.float64).tobytes())
    form = "gen" if kind == "diag" else kind   # a dense diagonal runs as a general 2x2 matrix
    r = subprocess.run([str(ix_check), "--apply", form, str(n), str(q), str(tmp_path / "psi.bin"),
                        str(tmp_path / "m.bin"), str(tmp_path / "out.bin")], capture_output=True, text=True)
    assert r.returncode == 0, r.stdout
    host = np.frombuffer((tmp_path / "out.bin").read_bytes(), dtype=np.complex128)
    idx = np.arange(1 << n, dtype=np.int64)
    gi = ((idx >> (q + 1)) << q) | (idx & ((1 << q) - 1))
    native = ((gi >> 8) % IX_GROUPS_PER_THREAD) < IX_NATIVE_GROUPS
    want = np.where(native, nat, host)
    bad = got.view(np.uint64).reshape(-1, 2) != want.view(np.uint64).reshape(-1, 2)
    bad = bad.any(axis=1)
    assert not bad.any(), (int(bad.sum()), int((bad & native).sum()), float(np.max(np.abs(got - want))))
    assert np.max(np.abs(got - nat)) <= 1e-15
