"""GPU parity of merged diagonal runs (phase-function passes) against the FP64 oracle:
fully connected and 3-regular QAOA, and random runs of RZ / Z / S / T / P / CZ / CP / RZZ
with few distinct angles on random qubits (lane, register and high index bits)."""
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


def run(qs, n, dtype, psi0, gates, **kw):
    h = qs.qs_create(n, dtype)
    try:
        qs.qs_set_amplitudes(h, psi0)
        qs.qs_apply_circuit(h, gates, qs.options(**kw))
        return qs.qs_amplitudes(h).astype(np.complex128), qs.qs_last_stats(h)
    finally:
        qs.qs_destroy(h)


def tol(dtype):
    return TOL_C128 if dtype == 2 else TOL_C64


def diag_runs(n, seed, layers=4, per_layer=40, angles=(0.3, 1.1)):
    r = np.random.default_rng(seed)
    names = ["rz", "z", "s", "t", "p", "cz", "cp", "rzz"]
    gates = []
    for _ in range(layers):
        gates += [("h", (q,), ()) for q in range(n)]
        for _ in range(per_layer):
            name = names[int(r.integers(len(names)))]
            k = inputs.arity(name)
            qubits = tuple(int(x) for x in r.choice(n, size=k, replace=False))
            params = (float(angles[int(r.integers(len(angles)))]),) if inputs.n_params(name) else ()
            gates.append((name, qubits, params))
    return gates


@pytest.mark.parametrize("dtype", [2, 1])
@pytest.mark.parametrize("n,m", [(12, 6), (16, 8), (18, 8)])
def test_complete_qaoa(qs, n, m, dtype):
    gates = inputs.qaoa_complete(n, p=3, seed=n)
    psi0 = oracle.zero_state(n)
    want = oracle.run(psi0.copy(), n, gates)
    p0 = psi0.astype(np.complex64 if dtype == 1 else np.complex128)
    got, st = run(qs, n, dtype, p0, gates, chunk_m=m)
    ref, st_n = run(qs, n, dtype, p0, gates, chunk_m=m, flags=qs.QS_OPT_NO_DIAG_MERGE)
    assert np.max(np.abs(got - want)) <= tol(dtype)
    assert np.max(np.abs(ref - want)) <= tol(dtype)
    assert st["passes"] < st_n["passes"]
    if dtype == 1:
        assert fidelity_gap(got, want) <= 1e-6


@pytest.mark.parametrize("dtype", [2, 1])
@pytest.mark.parametrize("n", [14, 17])
def test_regular_qaoa(qs, n, dtype):
    gates = inputs.qaoa_3regular(n, p=3, seed=2)
    psi0 = inputs.gaussian_state(n, seed=n)
    want = oracle.run(psi0.copy(), n, gates)
    p0 = psi0.astype(np.complex64 if dtype == 1 else np.complex128)
    got, _ = run(qs, n, dtype, p0, gates, chunk_m=7)
    assert np.max(np.abs(got - want)) <= tol(dtype)


@pytest.mark.parametrize("dtype", [2, 1])
@pytest.mark.parametrize("n,seed", [(9, 1), (13, 2), (16, 3), (19, 4)])
def test_random_diagonal_runs(qs, n, seed, dtype):
    gates = diag_runs(n, seed)
    psi0 = inputs.gaussian_state(n, seed=seed)
    want = oracle.run(psi0.copy(), n, gates)
    p0 = psi0.astype(np.complex64 if dtype == 1 else np.complex128)
    got, st = run(qs, n, dtype, p0, gates, chunk_m=6)
    assert np.max(np.abs(got - want)) <= tol(dtype)


def test_many_distinct_angles_stay_unmerged_and_exact(qs):
    """A run whose factors do not fit one table (every CP a different angle) is left to the
    ordinary passes; results are unchanged."""
    n = 15
    r = np.random.default_rng(9)
    gates = [("h", (q,), ()) for q in range(n)]
    for _ in range(80):
        a, b = (int(x) for x in r.choice(n, 2, replace=False))
        gates.append(("cp", (a, b), (float(r.uniform(0, 6.28)),)))
    psi0 = oracle.zero_state(n)
    want = oracle.run(psi0.copy(), n, gates)
    got, _ = run(qs, n, 2, psi0, gates, chunk_m=6)
    assert np.max(np.abs(got - want)) <= TOL_C128
