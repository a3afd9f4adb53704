"""Pins for the CPU oracle: values fixed by QueenV2's equations and by mathematics.

None of these re-types the oracle's own formulas.  Gate matrices are checked
against matrix exponentials of Pauli generators, textbook identities and the
CNOT matrix printed as Eq. 3; the gather/scatter update (Eq. 2 / Eq. 3) against
full Kronecker-product unitaries; whole circuits against closed forms (uniform
H^n|0>, GHZ, the QFT = inverse DFT, product states, QAOA bit-flip symmetry,
circuit followed by its inverse).
"""
import math
import os

import numpy as np
import pytest
from scipy.linalg import expm

import oracle
from paper_2409_14697_gb300 import inputs

HERE = os.path.dirname(os.path.abspath(__file__))
X = np.array([[0, 1], [1, 0]], dtype=complex)
Y = np.array([[0, -1j], [1j, 0]], dtype=complex)
Z = np.array([[1, 0], [0, -1]], dtype=complex)
I2 = np.eye(2, dtype=complex)
H_TEXTBOOK = np.array([[1, 1], [1, -1]], dtype=complex) / math.sqrt(2.0)


def rx(t):
    return expm(-0.5j * t * X)


def ry(t):
    return expm(-0.5j * t * Y)


def rz(t):
    return expm(-0.5j * t * Z)


def cnot_eq3():
    rows = [l.split() for l in open(os.path.join(HERE, "golden", "eq3_cnot.txt"))
            if l.strip() and not l.startswith("#")]
    return np.array(rows, dtype=float).astype(complex)


ANGLES = [0.0, 0.3, 1.1, math.pi / 2, 2.0, math.pi, 4.4, 5.9]


def test_cnot_is_eq3():
    assert np.array_equal(oracle.gate_matrix("cnot"), cnot_eq3())


def test_fixed_one_qubit_gates():
    assert np.allclose(oracle.gate_matrix("h"), H_TEXTBOOK, atol=1e-15)
    assert np.array_equal(oracle.gate_matrix("x"), X)
    assert np.array_equal(oracle.gate_matrix("y"), Y)
    assert np.array_equal(oracle.gate_matrix("z"), Z)
    s = oracle.gate_matrix("s")
    t = oracle.gate_matrix("t")
    assert np.allclose(s @ s, Z, atol=1e-15)
    assert np.allclose(t @ t, s, atol=1e-15)
    assert np.allclose(Y, 1j * X @ Z, atol=0)


@pytest.mark.parametrize("th", ANGLES)
def test_rotations_are_exponentials(th):
    assert np.allclose(oracle.gate_matrix("rx", (th,)), rx(th), atol=1e-14)
    assert np.allclose(oracle.gate_matrix("ry", (th,)), ry(th), atol=1e-14)
    assert np.allclose(oracle.gate_matrix("rz", (th,)), rz(th), atol=1e-14)
    assert np.allclose(oracle.gate_matrix("p", (th,)),
                       np.diag([1.0, np.exp(1j * th)]), atol=1e-15)
    zz = np.kron(Z, Z)
    assert np.allclose(oracle.gate_matrix("rzz", (th,)), expm(-0.5j * th * zz), atol=1e-14)


@pytest.mark.parametrize("seed", range(6))
def test_u3_is_zyz_euler(seed):
    t, ph, la = np.random.default_rng(seed).uniform(0, 2 * math.pi, 3)
    want = np.exp(0.5j * (ph + la)) * rz(ph) @ ry(t) @ rz(la)
    assert np.allclose(oracle.gate_matrix("u3", (t, ph, la)), want, atol=1e-14)


def test_u3_special_cases():
    assert np.allclose(oracle.gate_matrix("u3", (math.pi / 2, 0, math.pi)), H_TEXTBOOK, atol=1e-15)
    assert np.allclose(oracle.gate_matrix("u3", (math.pi, 0, math.pi)), X, atol=1e-15)
    for th in ANGLES:
        assert np.allclose(oracle.gate_matrix("u3", (th, -math.pi / 2, math.pi / 2)), rx(th), atol=1e-14)
        assert np.allclose(oracle.gate_matrix("u3", (th, 0, 0)), ry(th), atol=1e-14)
        assert np.allclose(oracle.gate_matrix("u3", (0, 0, th)),
                           np.exp(0.5j * th) * rz(th), atol=1e-14)


def test_two_qubit_identities():
    c01 = cnot_eq3()
    hh = np.kron(H_TEXTBOOK, H_TEXTBOOK)
    c10 = hh @ c01 @ hh            # conjugating by H(x)H swaps control and target
    ih = np.kron(I2, H_TEXTBOOK)
    assert np.allclose(oracle.gate_matrix("cz"), ih @ c01 @ ih, atol=1e-15)
    assert np.allclose(oracle.gate_matrix("swap"), c01 @ c10 @ c01, atol=1e-15)
    for th in ANGLES:
        assert np.allclose(oracle.gate_matrix("rzz", (th,)), c01 @ np.kron(I2, rz(th)) @ c01, atol=1e-14)
        assert np.allclose(oracle.gate_matrix("cp", (th,)),
                           np.diag([1, 1, 1, np.exp(1j * th)]), atol=1e-15)
    p0 = np.diag([1.0, 0.0]).astype(complex)
    p1 = np.diag([0.0, 1.0]).astype(complex)
    for seed in range(4):
        t, ph, la = np.random.default_rng(100 + seed).uniform(0, 2 * math.pi, 3)
        u = np.exp(0.5j * (ph + la)) * rz(ph) @ ry(t) @ rz(la)
        assert np.allclose(oracle.gate_matrix("cu3", (t, ph, la)),
                           np.kron(p0, I2) + np.kron(p1, u), atol=1e-14)
    assert np.allclose(np.kron(p0, I2) + np.kron(p1, X), c01, atol=0)


@pytest.mark.parametrize("name", [g for g in oracle.GATE_IDS if g != "dense"])
def test_unitary(name):
    m = oracle.gate_matrix(name, (0.7, 1.9, 4.1))
    assert np.allclose(m.conj().T @ m, np.eye(m.shape[0]), atol=1e-14)


def embed(n, qubits, g):
    """Full 2^n x 2^n operator of g on ``qubits`` (qubits[0] most significant in g's index),
    qubit 0 the right-most Kronecker factor.  Built as sum_{r,c} g[r,c] (x)_q E_q."""
    k = len(qubits)
    full = np.zeros((1 << n, 1 << n), dtype=complex)
    for r in range(1 << k):
        for c in range(1 << k):
            if g[r, c] == 0:
                continue
            term = np.ones((1, 1), dtype=complex)
            for q in reversed(range(n)):
                if q in qubits:
                    j = qubits.index(q)
                    br = (r >> (k - 1 - j)) & 1
                    bc = (c >> (k - 1 - j)) & 1
                    e = np.zeros((2, 2), dtype=complex)
                    e[br, bc] = 1.0
                else:
                    e = I2
                term = np.kron(term, e)
            full += g[r, c] * term
    return full


def gate_mat(gate):
    name, qubits, params = gate
    return np.asarray(params) if name == "dense" else oracle.gate_matrix(name, params)


@pytest.mark.parametrize("n,ng,seed", [(1, 10, 0), (2, 20, 1), (3, 30, 2), (4, 30, 3),
                                       (5, 40, 4), (7, 40, 5)])
def test_kronecker_brute_force(n, ng, seed):
    gates = inputs.random_circuit(n, ng, seed=seed)
    if n >= 3:   # dense 3-qubit and 2-qubit blocks on scattered operands
        gates.append(("dense", (2, 0, n - 1) if n > 3 else (2, 0, 1), inputs.random_unitary(3, seed)))
        gates.append(("dense", (n - 1, 1), inputs.random_unitary(2, seed)))
    psi0 = inputs.gaussian_state(n, seed=seed)
    u = np.eye(1 << n, dtype=complex)
    for g in gates:
        u = embed(n, list(g[1]), gate_mat(g)) @ u
    want = u @ psi0
    got = oracle.run(psi0.copy(), n, gates)
    assert np.max(np.abs(got - want)) < 1e-13


def test_eq2_pair_update_by_hand():
    # Eq. 2 on a 3-qubit basis: a gate on qubit 1 mixes exactly the pairs
    # (0,2), (1,3), (4,6), (5,7) of the basis index.
    g = np.array([[1, 2], [3, 4]], dtype=complex)
    psi = np.arange(8, dtype=complex) + 1j * np.arange(8)[::-1]
    want = psi.copy()
    for a, b in [(0, 2), (1, 3), (4, 6), (5, 7)]:
        want[a] = g[0, 0] * psi[a] + g[0, 1] * psi[b]
        want[b] = g[1, 0] * psi[a] + g[1, 1] * psi[b]
    got = psi.copy()
    oracle.apply_matrix(got, 3, [1], g)
    assert np.array_equal(got, want)


def test_eq3_cnot_on_basis_states():
    # CNOT(i=2 control, j=0 target) on |x>: flips bit 0 iff bit 2 is set.
    for x in range(16):
        psi = np.zeros(16, dtype=complex)
        psi[x] = 1
        oracle.run(psi, 4, [("cnot", (2, 0), ())])
        y = x ^ 1 if (x >> 2) & 1 else x
        assert psi[y] == 1 and np.count_nonzero(psi) == 1


def test_permutation_gates_on_basis_states():
    for x in range(32):
        psi = np.zeros(32, dtype=complex)
        psi[x] = 1
        oracle.run(psi, 5, [("x", (3,), ()), ("swap", (0, 4), ())])
        y = x ^ 8
        b0, b4 = y & 1, (y >> 4) & 1
        y = (y & ~0b10001) | (b0 << 4) | b4
        assert psi[y] == 1 and np.count_nonzero(psi) == 1


@pytest.mark.parametrize("n", [1, 5, 12])
def test_hadamard_all_uniform(n):
    psi = oracle.run(oracle.zero_state(n), n, [("h", (q,), ()) for q in range(n)])
    assert np.max(np.abs(psi - 2.0 ** (-n / 2))) < 1e-15
    assert np.allclose(oracle.expz(psi, n), 0.0, atol=1e-14)


@pytest.mark.parametrize("n", [2, 6, 11])
def test_ghz(n):
    gates = [("h", (0,), ())] + [("cnot", (q, q + 1), ()) for q in range(n - 1)]
    psi = oracle.run(oracle.zero_state(n), n, gates)
    want = np.zeros(1 << n, dtype=complex)
    want[0] = want[-1] = 1 / math.sqrt(2)
    assert np.max(np.abs(psi - want)) < 1e-15
    assert abs(oracle.norm(psi, n) - 1) < 1e-15
    assert np.allclose(oracle.expz(psi, n), 0.0, atol=1e-15)


@pytest.mark.parametrize("n", [3, 6, 9])
def test_qft_is_inverse_dft(n):
    gates = inputs.qft(n)
    for x in [0, 1, 5 % (1 << n), (1 << n) - 1]:
        psi = np.zeros(1 << n, dtype=complex)
        psi[x] = 1
        oracle.run(psi, n, gates)
        e = np.zeros(1 << n, dtype=complex)
        e[x] = 1
        assert np.max(np.abs(psi - np.fft.ifft(e) * math.sqrt(1 << n))) < 1e-13


def test_expz_basis_states():
    n = 6
    for x in [0, 1, 37, 63]:
        psi = np.zeros(1 << n, dtype=complex)
        psi[x] = 1j
        want = [1 - 2 * ((x >> i) & 1) for i in range(n)]
        assert np.array_equal(oracle.expz(psi, n), want)


def test_expz_product_state_closed_form():
    n = 7
    th = np.linspace(0.1, 3.0, n)
    psi = oracle.run(oracle.zero_state(n), n, [("ry", (q,), (th[q],)) for q in range(n)])
    assert np.allclose(oracle.expz(psi, n), np.cos(th), atol=1e-14)
    assert abs(oracle.norm(psi, n) - 1) < 1e-14


@pytest.mark.parametrize("n,layers", [(8, 5), (12, 20)])
def test_norm_and_inverse(n, layers):
    gates = inputs.brickwork(n, layers, seed=3)
    psi0 = inputs.gaussian_state(n, seed=4)
    psi = oracle.run(psi0.copy(), n, gates)
    assert abs(oracle.norm(psi, n) - 1) < 1e-13
    oracle.run(psi, n, inputs.inverse(gates))
    assert np.max(np.abs(psi - psi0)) < 1e-13


def test_inverse_of_every_gate_type():
    n = 4
    gates = inputs.random_circuit(n, 200, seed=11)
    psi0 = inputs.gaussian_state(n, seed=12)
    psi = oracle.run(psi0.copy(), n, gates + inputs.inverse(gates))
    assert np.max(np.abs(psi - psi0)) < 1e-13


def test_qaoa_bit_flip_symmetry():
    n = 10
    gates = inputs.qaoa_3regular(n, p=2, seed=1)
    psi = oracle.run(oracle.zero_state(n), n, gates)
    assert np.max(np.abs(psi - psi[::-1])) < 1e-14     # a_x = a_{not x}
    assert np.allclose(oracle.expz(psi, n), 0.0, atol=1e-14)


def test_tfim_limits():
    n, steps, dt = 6, 10, 0.05
    psi = oracle.run(oracle.zero_state(n), n, inputs.tfim(n, steps, dt, J=1.0, h=0.0))
    assert abs(abs(psi[0]) - 1) < 1e-14
    psi = oracle.run(oracle.zero_state(n), n, inputs.tfim(n, steps, dt, J=0.0, h=1.0))
    c, s = math.cos(dt * steps), 1j * math.sin(dt * steps)
    want = np.array([c ** (n - bin(x).count("1")) * s ** bin(x).count("1") for x in range(1 << n)])
    assert np.max(np.abs(psi - want)) < 1e-14


def test_top_k_order_and_ties():
    n = 5
    psi = np.zeros(32, dtype=complex)
    mags = [0.1, 0.5, 0.5, 0.3, 0.5j, 0.2]
    for i, m in zip([3, 7, 9, 12, 20, 31], mags):
        psi[i] = m
    idx, amp = oracle.top_k(psi, n, 5)
    assert list(idx) == [7, 9, 20, 12, 31]
    assert np.array_equal(amp, psi[idx.astype(np.int64)])


def test_random_3regular_degrees():
    for n in [10, 33]:
        edges = inputs.random_3regular(n)
        deg = np.zeros(n, dtype=int)
        for a, b in edges:
            assert a != b
            deg[a] += 1
            deg[b] += 1
        assert len(set(edges)) == len(edges)
        assert (deg[:n - (n % 2)] == 3).all() if n % 2 == 0 else \
            (sorted(deg)[0] == 2 and (np.sort(deg)[1:] == 3).all())
    assert len(inputs.random_3regular(33)) == 49


def test_oracle_rejects_bad_operands():
    psi = oracle.zero_state(3)
    with pytest.raises(ValueError):
        oracle.run(psi, 3, [("cnot", (1, 1), ())])
    with pytest.raises(ValueError):
        oracle.run(psi, 3, [("h", (3,), ())])


@pytest.mark.parametrize("n", [2, 6, 12, 16])
def test_threads_are_bitwise_equal_to_one_thread(n):
    """The threaded oracle (groups of a gate split over threads; whole subtrees of the
    pairwise sums handed to threads) gives the same bits as one thread: states after a
    mixed circuit with dense 3-qubit blocks, the norm and every <Z_q>."""
    psi0 = inputs.gaussian_state(n, seed=40 + n)
    gates = inputs.random_circuit(n, 60, seed=41)
    if n >= 3:
        gates += [("dense", (n - 1, 0, n // 2), inputs.random_unitary(3, seed=42))]
    gates += inputs.sweep_all(n, count=2)
    results = []
    before = oracle.threads()
    try:
        for t in (1, 3, 8):
            oracle.set_threads(t)
            a = oracle.run(psi0.copy(), n, gates)
            results.append((a, oracle.norm(a, n), oracle.expz(a, n)))
    finally:
        oracle.set_threads(before)
    a1, n1, e1 = results[0]
    assert abs(n1 - 1.0) < 1e-12
    for a, nr, ez in results[1:]:
        assert np.array_equal(a.view(np.uint64), a1.view(np.uint64))
        assert np.float64(nr).tobytes() == np.float64(n1).tobytes()
        assert np.array_equal(ez.view(np.uint64), e1.view(np.uint64))
