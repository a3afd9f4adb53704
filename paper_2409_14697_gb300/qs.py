"""Thin ctypes binding of the C interface in include/qs.h (argument marshalling only).

Every function keeps the C name (``qs_create``, ``qs_apply_circuit``, ...).  Gates
are passed either as ``qs_gate`` records or as ``(name, qubits, params)`` tuples
(``("dense", qubits, matrix)`` for a dense block), which :func:`gate_records`
converts.  Nothing here computes amplitudes: every step runs in ``libqsim.so``.
Importing this module fails loudly if the library has not been built.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libqsim.so")

QS_C64, QS_C128 = 1, 2
QS_OK, QS_NOT_READY = 0, 1
QS_ERR_INVALID, QS_ERR_NOMEM, QS_ERR_CUDA, QS_ERR_TIMEOUT, QS_ERR_BUSY, QS_ERR_UNSUPPORTED = -1, -2, -3, -4, -5, -6
QS_MODE_AUTO, QS_MODE_GATE, QS_MODE_CHUNK, QS_MODE_FUSED = 0, 1, 2, 3
QS_PREC_DEFAULT, QS_PREC_FP64, QS_PREC_DF32, QS_PREC_IX64 = 0, 1, 2, 3
QS_OPT_NO_REG_PHASES, QS_OPT_NO_DIAG_MERGE, QS_OPT_NO_TC_NORM_FIX, QS_OPT_NO_TPB = 1, 2, 4, 8
QS_REQ_BORROW_INIT = 1

GATE_TYPES = {
    "h": 0, "x": 1, "y": 2, "z": 3, "s": 4, "t": 5,
    "rx": 6, "ry": 7, "rz": 8, "p": 9, "u3": 10,
    "cnot": 11, "cz": 12, "swap": 13, "cu3": 14, "cp": 15, "rzz": 16,
    "dense": 17,
}


class QsError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"qs error {code}: {msg}")
        self.code = code


class qs_gate(ctypes.Structure):
    _fields_ = [("type", ctypes.c_int32), ("nq", ctypes.c_int32), ("q", ctypes.c_int32 * 8),
                ("p", ctypes.c_double * 3), ("m", ctypes.POINTER(ctypes.c_double))]


class qs_options(ctypes.Structure):
    _fields_ = [("mode", ctypes.c_int32), ("fuse_k", ctypes.c_int32), ("chunk_m", ctypes.c_int32),
                ("precision", ctypes.c_int32), ("flags", ctypes.c_uint32), ("reserved", ctypes.c_int32 * 4)]


class qs_stats(ctypes.Structure):
    _fields_ = [("gates_in", ctypes.c_int64), ("ops_after_fuse", ctypes.c_int64),
                ("passes", ctypes.c_int64), ("launches", ctypes.c_int64), ("bytes", ctypes.c_double),
                ("tile_sweeps", ctypes.c_int64), ("tc_blocks", ctypes.c_int64), ("tpb_gates", ctypes.c_int64),
                ("tc_flops", ctypes.c_double)]


class qs_circuit(ctypes.Structure):
    _fields_ = [("n_qubits", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("gates", ctypes.POINTER(qs_gate)), ("n_gates", ctypes.c_uint64)]


class qs_batch_stats(ctypes.Structure):
    _fields_ = [("circuits", ctypes.c_int64), ("passes", ctypes.c_int64), ("work_items", ctypes.c_int64),
                ("grid", ctypes.c_int64), ("state_bytes", ctypes.c_uint64)]


class qs_server_config(ctypes.Structure):
    _fields_ = [("hbm_budget_bytes", ctypes.c_uint64), ("max_slots", ctypes.c_int32),
                ("small_slots", ctypes.c_int32), ("small_max_qubits", ctypes.c_int32),
                ("reserved", ctypes.c_int32 * 3)]


class qs_request(ctypes.Structure):
    _fields_ = [("n_qubits", ctypes.c_int32), ("dtype", ctypes.c_int32),
                ("gates", ctypes.POINTER(qs_gate)), ("n_gates", ctypes.c_uint64),
                ("init_amplitudes", ctypes.c_void_p), ("top_k", ctypes.c_uint32), ("mode", ctypes.c_int32),
                ("precision", ctypes.c_int32), ("flags", ctypes.c_uint32)]


class qs_server_stats_t(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_int64), ("completed", ctypes.c_int64), ("failed", ctypes.c_int64),
                ("queued", ctypes.c_int64), ("in_flight", ctypes.c_int64),
                ("bytes_in_use", ctypes.c_uint64), ("peak_bytes", ctypes.c_uint64)]


_lib = None
_VP = ctypes.c_void_p
_DP = ctypes.POINTER(ctypes.c_double)
_U64P = ctypes.POINTER(ctypes.c_uint64)

# name -> (restype, argtypes)
_SIGS = {
    "qs_last_error": (ctypes.c_char_p, []),
    "qs_launch_count": (ctypes.c_uint64, []),
    "qs_version": (ctypes.c_int, [ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32)]),
    "qs_create": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.POINTER(_VP)]),
    "qs_create_on": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, _VP, ctypes.c_uint64, _VP, ctypes.POINTER(_VP)]),
    "qs_destroy": (ctypes.c_int, [_VP]),
    "qs_set_stream": (ctypes.c_int, [_VP, _VP]),
    "qs_synchronize": (ctypes.c_int, [_VP]),
    "qs_reset": (ctypes.c_int, [_VP]),
    "qs_info": (ctypes.c_int, [_VP, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(_VP)]),
    "qs_apply_circuit": (ctypes.c_int, [_VP, ctypes.POINTER(qs_gate), ctypes.c_size_t, ctypes.POINTER(qs_options)]),
    "qs_last_stats": (ctypes.c_int, [_VP, ctypes.POINTER(qs_stats)]),
    "qs_plan": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.POINTER(qs_gate), ctypes.c_size_t,
                               ctypes.POINTER(qs_options), ctypes.POINTER(ctypes.c_int32), _U64P,
                               ctypes.POINTER(ctypes.c_int64)]),
    "qs_set_amplitudes": (ctypes.c_int, [_VP, ctypes.c_uint64, ctypes.c_uint64, _VP]),
    "qs_amplitudes": (ctypes.c_int, [_VP, ctypes.c_uint64, ctypes.c_uint64, _VP]),
    "qs_set_amplitudes_async": (ctypes.c_int, [_VP, ctypes.c_uint64, ctypes.c_uint64, _VP]),
    "qs_amplitudes_async": (ctypes.c_int, [_VP, ctypes.c_uint64, ctypes.c_uint64, _VP]),
    "qs_norm": (ctypes.c_int, [_VP, _DP]),
    "qs_expectation_z": (ctypes.c_int, [_VP, _DP, _DP]),
    "qs_top_amplitudes": (ctypes.c_int, [_VP, ctypes.c_uint32, _U64P, _DP]),
    "qs_renormalize": (ctypes.c_int, [_VP, _DP]),
    "qs_expectation_z_noalloc": (ctypes.c_int, [_VP, ctypes.c_int, ctypes.c_int, _VP, _DP, _DP]),
    "qs_server_create": (ctypes.c_int, [ctypes.POINTER(qs_server_config), ctypes.POINTER(_VP)]),
    "qs_submit": (ctypes.c_int, [_VP, ctypes.POINTER(qs_request), ctypes.POINTER(ctypes.c_uint64)]),
    "qs_poll": (ctypes.c_int, [_VP, ctypes.c_uint64, _DP, _DP, _U64P, _DP, _DP]),
    "qs_server_stats": (ctypes.c_int, [_VP, ctypes.POINTER(qs_server_stats_t)]),
    "qs_server_drain": (ctypes.c_int, [_VP, ctypes.c_double]),
    "qs_server_destroy": (ctypes.c_int, [_VP]),
    "qs_batch_create": (ctypes.c_int, [ctypes.POINTER(qs_circuit), ctypes.c_size_t, ctypes.c_int,
                                       ctypes.POINTER(qs_options), ctypes.POINTER(_VP)]),
    "qs_batch_run": (ctypes.c_int, [_VP]),
    "qs_batch_synchronize": (ctypes.c_int, [_VP]),
    "qs_batch_set_stream": (ctypes.c_int, [_VP, _VP]),
    "qs_batch_amplitudes": (ctypes.c_int, [_VP, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint64, _VP]),
    "qs_batch_info": (ctypes.c_int, [_VP, ctypes.POINTER(qs_batch_stats)]),
    "qs_batch_destroy": (ctypes.c_int, [_VP]),
}


def load():
    """Loads libqsim.so (raises if it is missing: there is no fallback path)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is not built; run __graft_entry__.build()")
        lib = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


def exported_symbols():
    return list(_SIGS)


def _check(rc):
    if rc < 0:
        raise QsError(rc, load().qs_last_error().decode())
    return rc


def gate_records(gates):
    """(name, qubits, params) tuples -> ctypes array of qs_gate (dense matrices kept alive
    in the array's ``_keep`` attribute)."""
    arr = (qs_gate * max(len(gates), 1))()
    keep = []
    for i, (name, qubits, params) in enumerate(gates):
        g = arr[i]
        g.type = GATE_TYPES[name]
        g.nq = len(qubits)
        for j, q in enumerate(qubits):
            g.q[j] = int(q)
        if name == "dense":
            m = np.ascontiguousarray(params, dtype=np.complex128).reshape(-1).view(np.float64)
            keep.append(m)
            g.m = m.ctypes.data_as(_DP)
        else:
            for j, v in enumerate(params):
                g.p[j] = float(v)
    arr._keep = keep
    return arr


def options(mode=QS_MODE_AUTO, fuse_k=0, chunk_m=0, precision=QS_PREC_DEFAULT, flags=0):
    o = qs_options()
    o.mode, o.fuse_k, o.chunk_m, o.precision, o.flags = mode, fuse_k, chunk_m, precision, flags
    return o


# ---- C-named wrappers -----------------------------------------------------------

def qs_launch_count() -> int:
    return int(load().qs_launch_count())


def qs_version():
    a, d = ctypes.c_int32(), ctypes.c_int32()
    _check(load().qs_version(ctypes.byref(a), ctypes.byref(d)))
    return a.value, d.value


def qs_create(n_qubits: int, dtype: int = QS_C128):
    h = _VP()
    _check(load().qs_create(n_qubits, dtype, ctypes.byref(h)))
    return h


def qs_create_on(n_qubits: int, dtype: int, dev_ptr: int, nbytes: int, stream: int = 0):
    h = _VP()
    _check(load().qs_create_on(n_qubits, dtype, dev_ptr, nbytes, stream, ctypes.byref(h)))
    return h


def qs_destroy(h):
    _check(load().qs_destroy(h))


def qs_set_stream(h, stream: int):
    _check(load().qs_set_stream(h, stream))


def qs_synchronize(h):
    _check(load().qs_synchronize(h))


def qs_reset(h):
    _check(load().qs_reset(h))


def qs_info(h):
    n, d, p = ctypes.c_int32(), ctypes.c_int32(), _VP()
    _check(load().qs_info(h, ctypes.byref(n), ctypes.byref(d), ctypes.byref(p)))
    return n.value, d.value, p.value


def qs_apply_circuit(h, gates, opts=None):
    recs = gates if isinstance(gates, ctypes.Array) else gate_records(gates)
    n = len(gates)
    o = opts if opts is not None else options()
    _check(load().qs_apply_circuit(h, recs, n, ctypes.byref(o)))


def qs_last_stats(h) -> dict:
    s = qs_stats()
    _check(load().qs_last_stats(h, ctypes.byref(s)))
    return {f: getattr(s, f) for f, _ in qs_stats._fields_}


def qs_plan(n_qubits: int, dtype: int, gates, opts=None):
    """Host-only planner dry run: (pass index per gate, local-qubit mask per pass)."""
    recs = gates if isinstance(gates, ctypes.Array) else gate_records(gates)
    ng = len(gates)
    pog = np.zeros(max(ng, 1), dtype=np.int32)
    lm = np.zeros(max(ng, 1), dtype=np.uint64)
    npass = ctypes.c_int64()
    o = opts if opts is not None else options()
    _check(load().qs_plan(n_qubits, dtype, recs, ng, ctypes.byref(o),
                          pog.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), lm.ctypes.data_as(_U64P),
                          ctypes.byref(npass)))
    return pog[:ng], lm[:npass.value]


def _np_dtype(h):
    return np.complex128 if qs_info(h)[1] == QS_C128 else np.complex64


def qs_set_amplitudes(h, host: np.ndarray, off: int = 0):
    host = np.ascontiguousarray(host, dtype=_np_dtype(h))
    _check(load().qs_set_amplitudes(h, off, host.size, host.ctypes.data))


def qs_amplitudes(h, off: int = 0, cnt: int | None = None, out: np.ndarray | None = None):
    n = qs_info(h)[0]
    cnt = (1 << n) - off if cnt is None else cnt
    if out is None:
        out = np.empty(cnt, dtype=_np_dtype(h))
    _check(load().qs_amplitudes(h, off, cnt, out.ctypes.data))
    return out


def qs_amplitudes_into(h, off: int, cnt: int, host_ptr: int):
    _check(load().qs_amplitudes(h, off, cnt, host_ptr))


def qs_set_amplitudes_from(h, off: int, cnt: int, host_ptr: int):
    _check(load().qs_set_amplitudes(h, off, cnt, host_ptr))


def qs_set_amplitudes_async(h, off: int, cnt: int, host_ptr: int):
    """Stream-ordered host -> state copy; keep the buffer alive until qs_synchronize(h)."""
    _check(load().qs_set_amplitudes_async(h, off, cnt, host_ptr))


def qs_amplitudes_async(h, off: int, cnt: int, host_ptr: int):
    """Stream-ordered state -> host copy; read the buffer after qs_synchronize(h)."""
    _check(load().qs_amplitudes_async(h, off, cnt, host_ptr))


def qs_norm(h) -> float:
    v = ctypes.c_double()
    _check(load().qs_norm(h, ctypes.byref(v)))
    return v.value


def qs_expectation_z(h):
    n = qs_info(h)[0]
    out = np.zeros(n)
    nrm = ctypes.c_double()
    _check(load().qs_expectation_z(h, out.ctypes.data_as(_DP), ctypes.byref(nrm)))
    return out, nrm.value


def qs_top_amplitudes(h, k: int):
    idx = np.zeros(k, dtype=np.uint64)
    amp = np.zeros(k, dtype=np.complex128)
    _check(load().qs_top_amplitudes(h, k, idx.ctypes.data_as(_U64P), amp.ctypes.data_as(_DP)))
    return idx, amp


def qs_expectation_z_noalloc(dev_ptr: int, n_qubits: int, dtype: int, stream: int = 0):
    """Allocation-free <Z_q> and squared norm of a state at device address dev_ptr."""
    out = np.zeros(n_qubits)
    nrm = ctypes.c_double()
    _check(load().qs_expectation_z_noalloc(dev_ptr, n_qubits, dtype, stream, out.ctypes.data_as(_DP),
                                           ctypes.byref(nrm)))
    return out, nrm.value


def qs_renormalize(h) -> float:
    v = ctypes.c_double()
    _check(load().qs_renormalize(h, ctypes.byref(v)))
    return v.value


# ---- serving ----------------------------------------------------------------------

def qs_server_create(hbm_budget_bytes: int, max_slots: int = 8, small_slots: int = 0, small_max_qubits: int = 0):
    cfg = qs_server_config()
    cfg.hbm_budget_bytes = int(hbm_budget_bytes)
    cfg.max_slots = max_slots
    cfg.small_slots = small_slots
    cfg.small_max_qubits = small_max_qubits
    h = _VP()
    _check(load().qs_server_create(ctypes.byref(cfg), ctypes.byref(h)))
    return h


def qs_submit(sv, n_qubits: int, dtype: int, gates, top_k: int = 0, init=None, mode: int = QS_MODE_AUTO,
              precision: int = QS_PREC_DEFAULT, init_ptr: int = 0):
    """Queues a request; returns its ticket (the library copies gates and init).  init_ptr:
    host address of 2^n amplitudes that the request borrows (QS_REQ_BORROW_INIT): keep that
    buffer alive and unchanged until the ticket has been polled to completion."""
    recs = gates if isinstance(gates, ctypes.Array) else gate_records(gates)
    r = qs_request()
    r.n_qubits, r.dtype = n_qubits, dtype
    r.gates = ctypes.cast(recs, ctypes.POINTER(qs_gate))
    r.n_gates = len(gates)
    if init is not None:
        init = np.ascontiguousarray(init, dtype=np.complex64 if dtype == QS_C64 else np.complex128)
        r.init_amplitudes = init.ctypes.data
    elif init_ptr:
        r.init_amplitudes = init_ptr
        r.flags = QS_REQ_BORROW_INIT
    r.top_k, r.mode, r.precision = top_k, mode, precision
    t = ctypes.c_uint64()
    _check(load().qs_submit(sv, ctypes.byref(r), ctypes.byref(t)))
    return t.value


def qs_poll(sv, ticket: int, n_qubits: int, top_k: int):
    """None while running; else dict(expz, norm, top_idx, top_amp, latency_s)."""
    ez = np.zeros(max(n_qubits, 1))
    nrm = ctypes.c_double()
    idx = np.zeros(max(top_k, 1), dtype=np.uint64)
    amp = np.zeros(max(top_k, 1), dtype=np.complex128)
    lat = ctypes.c_double()
    rc = _check(load().qs_poll(sv, ticket, ez.ctypes.data_as(_DP), ctypes.byref(nrm), idx.ctypes.data_as(_U64P),
                               amp.ctypes.data_as(_DP), ctypes.byref(lat)))
    if rc == QS_NOT_READY:
        return None
    return {"expz": ez[:n_qubits], "norm": nrm.value, "top_idx": idx[:top_k], "top_amp": amp[:top_k],
            "latency_s": lat.value}


def qs_server_stats(sv) -> dict:
    s = qs_server_stats_t()
    _check(load().qs_server_stats(sv, ctypes.byref(s)))
    return {f: getattr(s, f) for f, _ in qs_server_stats_t._fields_}


def qs_server_drain(sv, timeout_s: float = 600.0):
    _check(load().qs_server_drain(sv, timeout_s))


def qs_server_destroy(sv):
    _check(load().qs_server_destroy(sv))


# ---- batched execution ----------------------------------------------------------

def qs_batch_create(circuits, dtype: int = QS_C64, opts=None):
    """circuits: list of (n_qubits, gates).  Returns an opaque batch handle."""
    arr = (qs_circuit * len(circuits))()
    keep = []
    for i, (n, gates) in enumerate(circuits):
        recs = gate_records(gates)
        keep.append(recs)
        arr[i].n_qubits = n
        arr[i].gates = ctypes.cast(recs, ctypes.POINTER(qs_gate))
        arr[i].n_gates = len(gates)
    h = _VP()
    o = opts if opts is not None else options()
    _check(load().qs_batch_create(arr, len(circuits), dtype, ctypes.byref(o), ctypes.byref(h)))
    return h


def qs_batch_run(b):
    _check(load().qs_batch_run(b))


def qs_batch_synchronize(b):
    _check(load().qs_batch_synchronize(b))


def qs_batch_set_stream(b, stream: int):
    _check(load().qs_batch_set_stream(b, stream))


def qs_batch_amplitudes(b, i: int, n: int, dtype: int = QS_C64):
    out = np.empty(1 << n, dtype=np.complex64 if dtype == QS_C64 else np.complex128)
    _check(load().qs_batch_amplitudes(b, i, 0, out.size, out.ctypes.data))
    return out


def qs_batch_info(b) -> dict:
    s = qs_batch_stats()
    _check(load().qs_batch_info(b, ctypes.byref(s)))
    return {f: getattr(s, f) for f, _ in qs_batch_stats._fields_}


def qs_batch_destroy(b):
    _check(load().qs_batch_destroy(b))


class State:
    """Owning wrapper: ``with State(n, QS_C128) as s: s.apply(gates)``."""

    def __init__(self, n: int, dtype: int = QS_C128):
        self.n, self.dtype = n, dtype
        self.h = qs_create(n, dtype)

    def apply(self, gates, mode=QS_MODE_AUTO, **kw):
        qs_apply_circuit(self.h, gates, options(mode=mode, **kw))
        return self

    def set(self, psi):
        qs_set_amplitudes(self.h, psi)
        return self

    def get(self):
        return qs_amplitudes(self.h)

    def sync(self):
        qs_synchronize(self.h)

    def close(self):
        if self.h:
            qs_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
