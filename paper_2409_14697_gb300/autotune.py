"""Autotuner for the planned path and the batched launch (host logic only).

The paper leaves the fusion decision to "a cost function" and notes that fusing 3 to 5
qubits is usually best (QueenV2 Sec. II-B).  Here the choice of chunk width m (local
qubits of an in-cache pass), fusion width k and the complex128 arithmetic is measured
instead of modelled: every candidate runs the real workload through the C ABI, timed with
CUDA events, and the fastest is kept.  Results are cached in a JSON file keyed by the
workload's signature (qubit count or range, dtype, gate mix), so a later run of the same
kind of workload reuses the choice without timing again.

The timing function is injectable, so the search and the cache are testable without a
GPU.  Nothing here touches amplitudes.
"""
from __future__ import annotations

import hashlib
import json
import os
import threading

DEFAULT_CACHE = os.path.join(os.path.expanduser("~"), ".cache", "qsim_gb300", "autotune.json")

_lock = threading.Lock()


def cache_path() -> str:
    return os.environ.get("QSIM_AUTOTUNE_CACHE", DEFAULT_CACHE)


def _load(path):
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _store(path, data):
    os.makedirs(os.path.dirname(path) or ".", exist_ok=True)
    tmp = f"{path}.tmp{os.getpid()}"
    with open(tmp, "w") as f:
        json.dump(data, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def signature(kind: str, n, dtype: int, gates_or_circuits) -> str:
    """Workload key: kind, qubit count (or range), dtype and a digest of the gate-type mix
    (counts per type, bucketed), not of the angles."""
    mix = {}
    if kind == "batch":
        for _, gates in gates_or_circuits:
            for g in gates:
                mix[g[0]] = mix.get(g[0], 0) + 1
    else:
        for g in gates_or_circuits:
            mix[g[0]] = mix.get(g[0], 0) + 1
    total = max(sum(mix.values()), 1)
    shape = sorted((k, round(v / total, 2)) for k, v in mix.items())
    digest = hashlib.sha1(json.dumps(shape).encode()).hexdigest()[:10]
    return f"{kind}|n={n}|dt={dtype}|mix={digest}|size={len(gates_or_circuits) // 64}"


def candidates(dtype: int, n: int, kind: str = "circuit"):
    """Candidate option sets: chunk width, fusion width (complex64: k = 1 applies gates
    unfused, in register phases on 2^13-amplitude tiles; tensor cores when k >= 4), and for
    complex128 the arithmetic (integer products, native FP64 or double-float)."""
    from . import qs
    out = []
    ms = [m for m in ((10, 11, 12) if dtype == qs.QS_C128 else (11, 12, 13)) if m <= max(n, 1)] or [0]
    if dtype == qs.QS_C128:
        precs = (qs.QS_PREC_FP64,) if kind == "batch" else (qs.QS_PREC_IX64, qs.QS_PREC_FP64, qs.QS_PREC_DF32)
        for m in ms:
            for prec in precs:
                for k in (1, 2):
                    out.append({"chunk_m": m, "fuse_k": k, "precision": prec})
    else:
        for m in ms:
            for k in (1, 2, 3, 4, 5, 6):
                if kind == "batch" and k > 4:
                    continue
                out.append({"chunk_m": m, "fuse_k": k, "precision": 0})
    return out


def search(key: str, cands, time_fn, path: str | None = None, force: bool = False):
    """Returns (best option dict, table of timings).  time_fn(option dict) -> ms; a
    candidate that raises is skipped.  The best is cached under key."""
    path = path or cache_path()
    with _lock:
        data = _load(path)
    if not force and key in data:
        return data[key]["best"], data[key]["table"]
    table = []
    for c in cands:
        try:
            ms = float(time_fn(c))
        except Exception as e:  # an option the workload cannot use
            table.append({**c, "ms": None, "error": str(e)[:120]})
            continue
        table.append({**c, "ms": ms})
    ok = [t for t in table if t["ms"] is not None]
    if not ok:
        raise RuntimeError("autotune: no candidate ran")
    best_row = min(ok, key=lambda t: t["ms"])
    best = {k: best_row[k] for k in ("chunk_m", "fuse_k", "precision")}
    with _lock:
        data = _load(path)
        data[key] = {"best": best, "table": table}
        _store(path, data)
    return best, table


def tune_circuit(n: int, dtype: int, gates, reps: int = 2, path: str | None = None, force: bool = False):
    """Best options for applying `gates` to an n-qubit state through qs_apply_circuit."""
    import torch

    from . import qs
    recs = qs.gate_records(gates)
    stream = torch.cuda.Stream()
    h = qs.qs_create(n, dtype)
    qs.qs_set_stream(h, stream.cuda_stream)

    def time_fn(c):
        o = qs.options(chunk_m=c["chunk_m"], fuse_k=c["fuse_k"], precision=c["precision"])
        qs.qs_apply_circuit(h, recs, o)      # warm-up, plans
        qs.qs_synchronize(h)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            qs.qs_apply_circuit(h, recs, o)
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps
    try:
        return search(signature("circuit", n, dtype, gates), candidates(dtype, n), time_fn, path, force)
    finally:
        qs.qs_destroy(h)


def tune_batch(circuits, dtype: int, reps: int = 2, path: str | None = None, force: bool = False):
    """Best chunk/fusion widths for one persistent launch over `circuits` [(n, gates)]."""
    import torch

    from . import qs
    stream = torch.cuda.Stream()
    n_lo = min(n for n, _ in circuits)
    n_hi = max(n for n, _ in circuits)

    def time_fn(c):
        b = qs.qs_batch_create(circuits, dtype, qs.options(chunk_m=c["chunk_m"], fuse_k=c["fuse_k"]))
        try:
            qs.qs_batch_set_stream(b, stream.cuda_stream)
            qs.qs_batch_run(b)
            qs.qs_batch_synchronize(b)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(reps):
                qs.qs_batch_run(b)
            e1.record(stream)
            qs.qs_batch_synchronize(b)
            return e0.elapsed_time(e1) / reps
        finally:
            qs.qs_batch_destroy(b)
    cands = [c for c in candidates(dtype, n_hi, "batch") if c["chunk_m"] >= 0]
    return search(signature("batch", f"{n_lo}-{n_hi}", dtype, circuits), cands, time_fn, path, force)
