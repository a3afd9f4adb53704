"""CPU tests of the chunk planner's host logic (qs_plan dry run, no GPU)."""
import numpy as np
import pytest

from paper_2409_14697_gb300 import inputs, qs


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2409_14697_gb300 import build
    build.build()


DIAGONAL = {"z", "s", "t", "rz", "p", "cz", "cp", "rzz"}


def qmask(g):
    m = 0
    for q in g[1]:
        m |= 1 << q
    return m


def check_plan(n, dtype, gates, chunk_m=0):
    pog, lm = qs.qs_plan(n, dtype, gates, qs.options(chunk_m=chunk_m))
    m = chunk_m or (12 if dtype == qs.QS_C128 else 13)
    if dtype == qs.QS_C128 and not chunk_m:   # small complex128 states: about 64 tiles
        m = max(7, min(m, n - 6))
    m = min(m, n)
    c = min(4 if dtype == qs.QS_C128 else 5, m)
    assert len(pog) == len(gates)
    assert (pog >= 0).all() and (pog < len(lm)).all()
    # every gate of a chunk pass lies inside the pass's local qubits, except that complex128
    # passes take two-qubit diagonals with one qubit outside (a per-tile factor on the other)
    for i, g in enumerate(gates):
        L = int(lm[pog[i]])
        if L:
            if dtype == qs.QS_C128 and g[0] in DIAGONAL and len(g[1]) == 2:
                assert qmask(g) & L, (i, g)
            else:
                assert qmask(g) & ~L == 0, (i, g)
            assert bin(L).count("1") == m
            assert L & ((1 << c) - 1) == (1 << c) - 1
    _deps_in_order(gates, pog)
    return pog, lm


@pytest.mark.parametrize("n", [6, 12, 20, 30, 33])
@pytest.mark.parametrize("dtype", [qs.QS_C128, qs.QS_C64])
def test_brickwork_plan_valid(n, dtype):
    gates = inputs.brickwork(n, 10, seed=1)
    pog, lm = check_plan(n, dtype, gates)
    m = 13 if dtype == qs.QS_C64 else max(7, min(12, n - 6))
    if n <= m:
        assert len(lm) == 1           # the whole state is one tile: one pass
    else:
        assert len(lm) < len(gates) / 4


@pytest.mark.parametrize("n", [14, 25, 33])
def test_qaoa_tfim_qft_plans_valid(n):
    for gates in (inputs.qaoa_3regular(n, p=2), inputs.tfim(n, steps=5), inputs.qft(min(n, 20))):
        check_plan(min(n, 20) if len(gates) and max(max(g[1]) for g in gates) < 20 else n,
                   qs.QS_C64, gates)


def test_random_and_dense_plans_valid():
    n = 18
    gates = inputs.random_circuit(n, 300, seed=3)
    gates.insert(50, ("dense", (17, 3, 9, 1, 0), inputs.random_unitary(5, 1)))
    gates.insert(120, ("dense", (2, 16), inputs.random_unitary(2, 2)))
    pog, lm = check_plan(n, qs.QS_C128, gates, chunk_m=10)
    assert lm[pog[50]] == 0           # a 5-qubit dense block is streamed on its own
    assert (pog == pog[50]).sum() == 1


def test_plan_rejects_invalid():
    with pytest.raises(qs.QsError):
        qs.qs_plan(4, qs.QS_C128, [("cz", (0, 4), ())])


@pytest.mark.parametrize("dtype", [qs.QS_C128, qs.QS_C64])
@pytest.mark.parametrize("n,m", [(8, 6), (8, 5), (10, 4), (14, 6), (6, 6)])
def test_small_chunk_width_always_progresses(n, m, dtype):
    """With few free local slots some ops cannot join any pass: they are streamed, and
    the planner still assigns every gate exactly once (no empty passes)."""
    gates = inputs.random_circuit(n, 200, seed=n + m) + inputs.brickwork(n, 6, seed=n)
    pog, lm = check_plan(n, dtype, gates, chunk_m=m)
    assert len(lm) <= len(gates)
    counts = np.bincount(pog, minlength=len(lm))
    assert (counts >= 1).all()


def test_window_search_cuts_passes():
    """The windowed local-set search executes brickwork and TFIM chains in far fewer
    passes than claiming local qubits in circuit order (85 / 197 before the search)."""
    g = inputs.brickwork(33, 40, seed=3)
    pog, lm = check_plan(33, qs.QS_C64, g)
    assert len(lm) <= 40
    g = inputs.tfim(33, 50)
    pog, lm = check_plan(33, qs.QS_C64, g)
    assert len(lm) <= 90


@pytest.mark.parametrize("n", [23, 30])
def test_qft_controlled_phases_with_nonlocal_qubit(n):
    """complex128 passes take a target's controlled phases whatever its partner's position
    (a per-tile factor when the partner is outside the local set), so each pass takes the
    next 8 Hadamard targets: 30 qubits need 6 passes instead of 35; complex64 keeps the old
    rule (register phases hold local gates only)."""
    gates = inputs.qft(n)
    pog, lm = check_plan(n, qs.QS_C128, gates)
    assert len(lm) <= (4 if n == 23 else 6)
    pog64, lm64 = check_plan(n, qs.QS_C64, gates)
    assert len(lm64) > 2 * len(lm)


def test_nonlocal_diagonals_only_controlled_phases():
    """RZZ (no control) stays a local-only gate; CP, CZ and CU3(0, ..) may leave one qubit
    outside the pass."""
    n = 20
    r = np.random.default_rng(4)
    gates = [("h", (q,), ()) for q in range(n)]
    for _ in range(200):
        a, b = (int(x) for x in r.choice(n, 2, replace=False))
        gates.append(("rzz", (a, b), (0.3,)))
    pog, lm = qs.qs_plan(n, qs.QS_C128, gates, qs.options(chunk_m=8, flags=qs.QS_OPT_NO_DIAG_MERGE))
    for (name, qb, _), p in zip(gates, pog):
        L = int(lm[p])
        if L:
            assert qmask((name, qb, ())) & ~L == 0


def _deps_in_order(gates, pog):
    """Gates sharing a qubit keep their pass order unless both are diagonal (diagonal gates
    commute with each other, so the planner may run a later one in an earlier pass)."""
    last_any, last_nondiag = {}, {}
    for i, g in enumerate(gates):
        d = g[0] in DIAGONAL
        for q in g[1]:
            # this gate must not run before any earlier non-diagonal gate on q, and a
            # non-diagonal gate not before any earlier gate on q
            ref = last_nondiag.get(q) if d else last_any.get(q)
            if ref is not None:
                assert pog[ref] <= pog[i], (i, g, ref, gates[ref])
        for q in g[1]:
            if not d:
                last_nondiag[q] = i
            # the latest gate on q that a later non-diagonal gate must follow
            if not d or q not in last_any or pog[i] >= pog[last_any[q]]:
                last_any[q] = i


def test_diag_merge_cuts_passes_for_complete_qaoa():
    """Fully connected QAOA: each layer's equal-angle RZZ run becomes one phase-function
    pass (merged plan), far fewer passes than packing all-pairs RZZ into chunk passes."""
    n = 22
    gates = inputs.qaoa_complete(n, p=2, seed=1)
    # complex64 passes hold only local gates: merging saves passes
    pog_m, lm_m = qs.qs_plan(n, qs.QS_C64, gates)
    pog_n, lm_n = qs.qs_plan(n, qs.QS_C64, gates, qs.options(flags=qs.QS_OPT_NO_DIAG_MERGE))
    assert len(lm_m) < len(lm_n)
    _deps_in_order(gates, pog_m)
    # complex128 passes also take RZZ with a non-local qubit; at equal pass counts the merged
    # runs (one table lookup per amplitude) are kept
    pog_m, lm_m = qs.qs_plan(n, qs.QS_C128, gates)
    pog_n, lm_n = qs.qs_plan(n, qs.QS_C128, gates, qs.options(flags=qs.QS_OPT_NO_DIAG_MERGE))
    assert len(lm_m) <= len(lm_n)
    _deps_in_order(gates, pog_m)
    # the RZZ gates of one layer share one streamed pass (no local mask)
    npairs = n * (n - 1) // 2
    start = n
    for _ in range(2):
        layer = pog_m[start:start + npairs]
        assert (layer == layer[0]).all()
        assert int(lm_m[layer[0]]) == 0
        start += npairs + n


def test_diag_merge_not_taken_for_tfim_chain():
    """TFIM: chunk passes follow the chain's light cone; merging each RZZ layer into a
    full-state pass would need more passes, so the plain plan is kept."""
    n = 24
    gates = inputs.tfim(n, steps=10)
    _, lm_m = qs.qs_plan(n, qs.QS_C64, gates)
    _, lm_n = qs.qs_plan(n, qs.QS_C64, gates, qs.options(flags=qs.QS_OPT_NO_DIAG_MERGE))
    assert len(lm_m) == len(lm_n)


def test_diag_merge_respects_non_diagonal_barriers():
    """A merged run never crosses a non-diagonal gate: gates before and after it on the
    same qubits keep their order."""
    n = 20
    r = np.random.default_rng(3)
    gates = []
    for layer in range(6):
        gates += [("h", (q,), ()) for q in range(n)]
        for _ in range(30):
            a, b = (int(x) for x in r.choice(n, 2, replace=False))
            gates.append(("rzz", (a, b), (0.7,)))
    pog, lm = qs.qs_plan(n, qs.QS_C64, gates, qs.options(chunk_m=8))
    _deps_in_order(gates, pog)
