"""GPU tests of the serving runtime: oracle parity of every result, bitwise identical
results alone and in a concurrent mix, admission by HBM budget, and the error paths."""
import time

import numpy as np
import pytest

import oracle
from paper_2409_14697_gb300 import inputs
from tests.gpu_util import TOL_C128, TOL_C64, require_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def qs():
    require_gpu()
    from paper_2409_14697_gb300 import qs as q
    q.load()
    return q


def wait(qs, sv, t, n, k, timeout=120.0):
    t0 = time.time()
    while True:
        r = qs.qs_poll(sv, t, n, k)
        if r is not None:
            return r
        assert time.time() - t0 < timeout
        time.sleep(0.0005)


def make_requests(count, seed):
    reqs = inputs.served_stream(count, rate_hz=2000.0, seed=seed, n_range=(10, 20))
    out = []
    for r in reqs:
        init = inputs.gaussian_state(r["n"], seed=r["init_seed"]) if r["init_seed"] else None
        out.append((r["n"], 2 if r["dtype"] == "c128" else 1, r["gates"], init))
    return out


def test_results_match_oracle_and_are_mix_independent(qs):
    reqs = make_requests(24, seed=1)
    k = 64
    sv = qs.qs_server_create(8 << 30, max_slots=6)
    try:
        # all at once (a concurrent mix)
        tickets = [qs.qs_submit(sv, n, dt, g, top_k=k, init=init) for n, dt, g, init in reqs]
        mixed = [wait(qs, sv, t, n, k) for t, (n, dt, g, init) in zip(tickets, reqs)]
        # each alone
        alone = []
        for n, dt, g, init in reqs:
            t = qs.qs_submit(sv, n, dt, g, top_k=k, init=init)
            alone.append(wait(qs, sv, t, n, k))
        st = qs.qs_server_stats(sv)
        assert st["completed"] == 2 * len(reqs) and st["failed"] == 0
        assert st["peak_bytes"] <= 8 << 30
    finally:
        qs.qs_server_drain(sv)
        qs.qs_server_destroy(sv)
    for (n, dt, g, init), a, b in zip(reqs, mixed, alone):
        # bitwise the same alone and in the mix
        assert np.array_equal(a["expz"], b["expz"]) and a["norm"] == b["norm"]
        assert np.array_equal(a["top_idx"], b["top_idx"]) and np.array_equal(a["top_amp"], b["top_amp"])
        psi0 = oracle.zero_state(n) if init is None else init.astype(np.complex64 if dt == 1 else np.complex128).astype(np.complex128)
        want = oracle.run(psi0.copy(), n, g)
        tol = 1e-12 if dt == 2 else 1e-5
        assert np.max(np.abs(a["expz"] - oracle.expz(want, n))) <= tol
        assert abs(a["norm"] - oracle.norm(want, n)) <= tol
        # top-k: probabilities at the returned indices are the largest (within tolerance)
        p = np.abs(want) ** 2
        kth = np.sort(p)[-k]
        got_p = p[a["top_idx"].astype(np.int64)]
        assert np.all(got_p >= kth - (1e-12 if dt == 2 else 1e-6))
        assert np.max(np.abs(a["top_amp"] - want[a["top_idx"].astype(np.int64)])) <= (TOL_C128 if dt == 2 else TOL_C64)


def test_admission_respects_budget(qs):
    # budget for two 20-qubit complex128 states at a time
    budget = 2 * (16 << 20)
    sv = qs.qs_server_create(budget, max_slots=8)
    try:
        gates = inputs.brickwork(20, 4, seed=2)
        tickets = [qs.qs_submit(sv, 20, 2, gates, top_k=4) for _ in range(6)]
        for t in tickets:
            wait(qs, sv, t, 20, 4)
        st = qs.qs_server_stats(sv)
        assert st["peak_bytes"] <= budget
        with pytest.raises(qs.QsError) as e:       # can never fit
            qs.qs_submit(sv, 22, 2, gates[:1])
        assert e.value.code == qs.QS_ERR_NOMEM
    finally:
        qs.qs_server_drain(sv)
        qs.qs_server_destroy(sv)


def test_error_paths(qs):
    sv = qs.qs_server_create(1 << 30, max_slots=2)
    try:
        with pytest.raises(qs.QsError) as e:
            qs.qs_poll(sv, 12345, 4, 0)
        assert e.value.code == qs.QS_ERR_INVALID
        with pytest.raises(qs.QsError) as e:
            qs.qs_submit(sv, 4, 2, [("cnot", (1, 1), ())])
        assert e.value.code == qs.QS_ERR_INVALID
        t = qs.qs_submit(sv, 24, 1, inputs.brickwork(24, 10, seed=3), top_k=8)
        with pytest.raises(qs.QsError) as e:        # still in flight
            qs.qs_server_destroy(sv)
        assert e.value.code == qs.QS_ERR_BUSY
        wait(qs, sv, t, 24, 8)
        with pytest.raises(qs.QsError):              # a ticket is returned once
            qs.qs_poll(sv, t, 24, 8)
    finally:
        qs.qs_server_drain(sv)
        qs.qs_server_destroy(sv)


def test_borrowed_initial_amplitudes(qs):
    """Requests that borrow the caller's initial amplitudes (QS_REQ_BORROW_INIT, no copy at
    submission): several requests share one page-locked buffer and one pageable buffer;
    results are bitwise those of requests whose amplitudes were copied, and match the
    oracle."""
    torch = pytest.importorskip("torch")
    n, k = 18, 16
    psi = inputs.gaussian_state(n, seed=77)
    pinned = torch.empty(psi.view(np.float64).size, dtype=torch.float64, pin_memory=True)
    pinned.numpy()[:] = psi.view(np.float64)
    pageable = psi.copy()
    circuits = [inputs.gate_sweep(n, g, seed=9, count=30) for g in ("u3", "cnot", "h", "cu3")]
    sv = qs.qs_server_create(4 << 30, max_slots=4)
    try:
        tickets = []
        for i, g in enumerate(circuits):
            ptr = pinned.data_ptr() if i % 2 == 0 else pageable.ctypes.data
            tickets.append(qs.qs_submit(sv, n, 2, g, top_k=k, init_ptr=ptr))
        borrowed = [wait(qs, sv, t, n, k) for t in tickets]
        copied = [wait(qs, sv, qs.qs_submit(sv, n, 2, g, top_k=k, init=psi), n, k) for g in circuits]
        with pytest.raises(qs.QsError) as e:          # unknown flag bits are rejected
            r = qs.qs_request()
            r.n_qubits, r.dtype, r.flags = n, 2, 8
            t = qs.ctypes.c_uint64()
            qs._check(qs.load().qs_submit(sv, qs.ctypes.byref(r), qs.ctypes.byref(t)))
        assert e.value.code == qs.QS_ERR_INVALID
    finally:
        qs.qs_server_drain(sv)
        qs.qs_server_destroy(sv)
    for g, a, b in zip(circuits, borrowed, copied):
        assert np.array_equal(a["expz"], b["expz"]) and a["norm"] == b["norm"]
        assert np.array_equal(a["top_idx"], b["top_idx"]) and np.array_equal(a["top_amp"], b["top_amp"])
        want = oracle.run(psi.copy(), n, g)
        assert np.max(np.abs(a["expz"] - oracle.expz(want, n))) <= 1e-12


def test_small_requests_overtake_large_ones(qs):
    """One regular slot, held by large requests, and a small lane of two slots: small
    requests submitted after two large ones start at once and finish before the first large
    one (whose kernels run meanwhile; the small lane's streams have the higher priority), and
    the second large one waits for the first (large ones keep their order).  Results are
    those of the oracle, and the large ones' those of the plain entry points bit for bit."""
    n_big, k = 26, 8
    big = inputs.brickwork(n_big, 60, seed=1)
    sv = qs.qs_server_create(8 << 30, max_slots=1, small_slots=2, small_max_qubits=12)
    try:
        # first use of the server's slots and streams, alone (the first requests of a fresh
        # server were measured not to overlap)
        for n, dt, g in ((n_big, 2, big), (10, 1, inputs.brickwork(10, 2, seed=99)),
                         (10, 1, inputs.brickwork(10, 2, seed=98))):
            wait(qs, sv, qs.qs_submit(sv, n, dt, g, top_k=k), n, k)
        t_big = [qs.qs_submit(sv, n_big, 2, big, top_k=k) for _ in range(2)]
        smalls = [(10 + (i % 3), inputs.brickwork(10 + (i % 3), 20, seed=100 + i)) for i in range(6)]
        t_small = [qs.qs_submit(sv, n, 1, g, top_k=k) for n, g in smalls]
        r_small = [wait(qs, sv, t, n, k) for t, (n, g) in zip(t_small, smalls)]
        r_big = [wait(qs, sv, t, n_big, k) for t in t_big]
    finally:
        qs.qs_server_drain(sv)
        qs.qs_server_destroy(sv)
    assert r_big[0]["latency_s"] < r_big[1]["latency_s"]
    assert max(r["latency_s"] for r in r_small) < r_big[0]["latency_s"], \
        ([r["latency_s"] for r in r_small], r_big[0]["latency_s"])
    assert np.array_equal(r_big[0]["expz"], r_big[1]["expz"])
    # the large requests ran as grids of short-lived blocks (a small lane is configured):
    # bitwise the results of the same circuit through the plain entry points
    h = qs.qs_create(n_big, 2)
    try:
        qs.qs_apply_circuit(h, big)
        ez, nrm = qs.qs_expectation_z(h)
    finally:
        qs.qs_destroy(h)
    assert np.array_equal(r_big[0]["expz"], ez) and r_big[0]["norm"] == nrm
    for (n, g), r in zip(smalls, r_small):
        want = oracle.run(oracle.zero_state(n), n, g)
        assert np.max(np.abs(r["expz"] - oracle.expz(want, n))) <= 1e-5


def test_server_rejects_bad_small_lane(qs):
    with pytest.raises(qs.QsError) as e:
        qs.qs_server_create(1 << 30, max_slots=2, small_slots=-1)
    assert e.value.code == qs.QS_ERR_INVALID
