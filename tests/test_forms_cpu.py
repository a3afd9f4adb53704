"""CPU pins of the exact algebraic forms the GPU executor applies in place of some gates,
checked against the oracle's own gate matrices (the executor's results are compared with
the oracle element by element in the GPU tests; these pin the identities themselves):

* RZ(theta) = e^{-i theta/2} diag(1, e^{i theta}): gate-by-gate calls apply the diagonal on
  the half with the target bit set and carry the global phases to the call's last RZ;
* H = 2^{-1/2} (a + b, a - b): the unscaled butterflies of a call or pass and one scaled
  one carrying 2^{-k/2} give the same state as k Hadamards;
* U3(theta, phi, lambda) = P(phi) R P(lambda) with R = [[c, -s], [s, c]] real, P(x) =
  diag(1, e^{ix}): complex128 FP64 passes apply R and merge the phases with neighbouring
  diagonals;
* a two-qubit diagonal d(x_a, x_h) = d(x_a, 0) [x_h ? d(x_a, 1)/d(x_a, 0) : 1], which for a
  controlled phase (d(0, x) = 1) is a phase on a's 1-half chosen by the bit x_h: the form a
  chunk pass uses when x_h is outside its tile.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2409_14697_gb300 import inputs

pytestmark = pytest.mark.filterwarnings("ignore")


def P(x):
    return np.diag([1.0, np.exp(1j * x)])


@pytest.mark.parametrize("seed", range(6))
def test_rz_is_global_phase_times_phase_gate(seed):
    th = float(np.random.default_rng(seed).uniform(0, 4 * math.pi))
    rz = oracle.gate_matrix("rz", (th,))
    assert np.allclose(rz, np.exp(-0.5j * th) * P(th), atol=1e-15)
    # the factored phases of many RZ multiply into the last one: a product of RZ on one
    # qubit equals the product of the phase forms times the product of the phases
    r = np.random.default_rng(100 + seed)
    ths = r.uniform(0, 2 * math.pi, 7)
    prod = np.eye(2, dtype=complex)
    folded = np.eye(2, dtype=complex)
    g = 1.0 + 0j
    for t in ths:
        prod = oracle.gate_matrix("rz", (float(t),)) @ prod
        folded = P(float(t)) @ folded
        g *= np.exp(-0.5j * t)
    assert np.allclose(prod, g * folded, atol=1e-14)


@pytest.mark.parametrize("n,k", [(3, 3), (5, 4), (6, 9)])
def test_unscaled_hadamards_with_one_scaled(n, k):
    """k Hadamards on random qubits: k - 1 unscaled butterflies and the last scaled by
    2^{-k/2} give the oracle's state."""
    r = np.random.default_rng(n * 10 + k)
    qs = [int(q) for q in r.integers(0, n, k)]
    psi0 = inputs.gaussian_state(n, seed=n + k)
    want = oracle.run(psi0.copy(), n, [("h", (q,), ()) for q in qs])
    got = psi0.copy()
    butterfly = np.array([[1.0, 1.0], [1.0, -1.0]], dtype=complex)
    for i, q in enumerate(qs):
        scale = 2.0 ** (-k / 2) if i == k - 1 else 1.0
        oracle.apply_matrix(got, n, (q,), scale * butterfly)
    assert np.max(np.abs(got - want)) <= 1e-14


@pytest.mark.parametrize("seed", range(8))
def test_u3_is_phase_rotation_phase(seed):
    t, ph, la = (float(x) for x in np.random.default_rng(seed).uniform(0, 2 * math.pi, 3))
    u3 = oracle.gate_matrix("u3", (t, ph, la))
    c, s = math.cos(t / 2), math.sin(t / 2)
    R = np.array([[c, -s], [s, c]])
    assert np.allclose(u3, P(ph) @ R @ P(la), atol=1e-15)
    # the executor's reading of the parts from the matrix itself (real first entry):
    # s = |u10|, e^{i phi} = u10 / s, e^{i lambda} = -u01 / s
    sv = abs(u3[1, 0])
    e_ph, e_la = u3[1, 0] / sv, -u3[0, 1] / sv
    R2 = np.array([[u3[0, 0].real, -sv], [sv, u3[0, 0].real]])
    assert np.allclose(np.diag([1, e_ph]) @ R2 @ np.diag([1, e_la]), u3, atol=1e-14)


@pytest.mark.parametrize("gate", ["cp", "cz", "rzz"])
def test_two_qubit_diagonal_split_by_one_bit(gate):
    """d(x_a, x_h) = d(x_a, 0) [x_h ? d(x_a, 1) / d(x_a, 0) : 1], and for controlled phases
    (d(0, x) = 1) the x_h part touches only a's 1-half."""
    params = (0.7,) if gate in ("cp", "rzz") else ()
    u = oracle.gate_matrix(gate, params)
    d = np.diag(u).reshape(2, 2)            # d[x_a, x_h], first operand = a
    for xa in (0, 1):
        for xh in (0, 1):
            f = d[xa, 1] / d[xa, 0] if xh else 1.0
            assert abs(d[xa, 0] * f - d[xa, xh]) <= 1e-15
    controlled = np.allclose(d[0, :], 1.0)
    assert controlled == (gate != "rzz")
