"""CPU tests of the autotuner's search and cache (timing function faked)."""
import pytest

from paper_2409_14697_gb300 import autotune, inputs, qs


def test_search_picks_fastest_and_caches(tmp_path):
    path = str(tmp_path / "cache.json")
    cands = [{"chunk_m": m, "fuse_k": k, "precision": 0} for m in (11, 12, 13) for k in (2, 4)]
    calls = []

    def fake(c):
        calls.append(c)
        if c["fuse_k"] == 4 and c["chunk_m"] == 11:
            raise RuntimeError("not supported")
        return abs(c["chunk_m"] - 12) * 10 + c["fuse_k"]
    best, table = autotune.search("k1", cands, fake, path)
    assert best == {"chunk_m": 12, "fuse_k": 2, "precision": 0}
    assert len(calls) == len(cands)
    assert any(t["ms"] is None for t in table)
    calls.clear()
    best2, _ = autotune.search("k1", cands, fake, path)      # cached: no timing
    assert best2 == best and not calls
    autotune.search("k1", cands, fake, path, force=True)      # forced: times again
    assert len(calls) == len(cands)


def test_search_raises_when_nothing_runs(tmp_path):
    def bad(c):
        raise RuntimeError("no")
    with pytest.raises(RuntimeError):
        autotune.search("k2", [{"chunk_m": 12, "fuse_k": 2, "precision": 0}], bad, str(tmp_path / "c.json"))


def test_signature_ignores_angles_but_not_gate_mix():
    a = autotune.signature("circuit", 20, 1, inputs.brickwork(20, 5, seed=1))
    b = autotune.signature("circuit", 20, 1, inputs.brickwork(20, 5, seed=2))
    c = autotune.signature("circuit", 20, 1, inputs.qaoa_3regular(20, p=2))
    assert a == b and a != c


def test_candidates_cover_both_dtypes():
    c128 = autotune.candidates(qs.QS_C128, 30)
    c64 = autotune.candidates(qs.QS_C64, 30)
    assert {c["precision"] for c in c128} == {qs.QS_PREC_IX64, qs.QS_PREC_FP64, qs.QS_PREC_DF32}
    assert max(c["fuse_k"] for c in c64) == 6
    assert min(c["fuse_k"] for c in c64) == 1
    assert all(c["fuse_k"] <= 4 for c in autotune.candidates(qs.QS_C64, 20, "batch"))
