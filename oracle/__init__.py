"""Plain FP64 CPU oracle for the state-vector simulator (test infrastructure).

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` import this package.  The product library never loads it.

``qs_oracle.c`` holds the arithmetic (Eq. 1-3 of QueenV2, arXiv 2409.14697,
applied gate by gate); this module compiles it with the host C compiler and
wraps it with ctypes.  Gates are described by the seeded generators in
``paper_2409_14697_gb300.inputs`` as ``(name, qubits, params)`` tuples, or as
``("dense", qubits, matrix)``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "qs_oracle.c")
_LIB = os.path.join(_HERE, "libqs_oracle.so")

# Gate ids as the oracle's C source numbers them.
GATE_IDS = {
    "h": 0, "x": 1, "y": 2, "z": 3, "s": 4, "t": 5,
    "rx": 6, "ry": 7, "rz": 8, "p": 9, "u3": 10,
    "cnot": 11, "cz": 12, "swap": 13, "cu3": 14, "cp": 15, "rzz": 16,
    "dense": 17,
}

_lib = None


def build(force: bool = False) -> str:
    """Compile ``qs_oracle.c`` into ``libqs_oracle.so`` (plain -O2; OpenMP when the
    compiler supports it, else one thread)."""
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    base = [os.environ.get("CC", "gcc"), "-O2", "-std=c99", "-fPIC", "-shared",
            "-fcx-limited-range", "-D_GNU_SOURCE", _SRC, "-o", tmp, "-lm"]
    r = subprocess.run(base[:1] + ["-fopenmp"] + base[1:], capture_output=True, text=True)
    if r.returncode != 0:
        subprocess.check_call(base)
    os.replace(tmp, _LIB)
    return _LIB


def default_threads() -> int:
    """Host threads the oracle uses unless told otherwise: QS_ORACLE_THREADS, else every
    core this process may run on."""
    env = os.environ.get("QS_ORACLE_THREADS")
    if env:
        return max(1, int(env))
    try:
        return max(1, len(os.sched_getaffinity(0)))
    except AttributeError:
        return max(1, os.cpu_count() or 1)


def set_threads(t: int) -> int:
    """Sets the oracle's thread count; returns the count in effect (1 without OpenMP).
    Results do not depend on it (bitwise)."""
    return int(_load().or_set_threads(int(t)))


def threads() -> int:
    return int(_load().or_get_threads())


def has_openmp() -> bool:
    return bool(_load().or_has_openmp())


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        dp = ctypes.POINTER(ctypes.c_double)
        ip = ctypes.POINTER(ctypes.c_int)
        lp = ctypes.POINTER(ctypes.c_long)
        u64p = ctypes.POINTER(ctypes.c_uint64)
        lib.or_gate_matrix.argtypes = [ctypes.c_int, dp, dp]
        lib.or_gate_matrix.restype = ctypes.c_int
        lib.or_apply_matrix.argtypes = [dp, ctypes.c_int, ctypes.c_int, ip, dp]
        lib.or_apply_matrix.restype = ctypes.c_int
        lib.or_run.argtypes = [dp, ctypes.c_int, ctypes.c_long, ip, ip, ip, dp, dp, lp]
        lib.or_run.restype = ctypes.c_int
        lib.or_zero_state.argtypes = [dp, ctypes.c_int]
        lib.or_norm.argtypes = [dp, ctypes.c_int]
        lib.or_norm.restype = ctypes.c_double
        lib.or_expz.argtypes = [dp, ctypes.c_int, dp]
        lib.or_top_k.argtypes = [dp, ctypes.c_int, ctypes.c_long, u64p, dp]
        lib.or_top_k.restype = ctypes.c_int
        lib.or_set_threads.argtypes = [ctypes.c_int]
        lib.or_set_threads.restype = ctypes.c_int
        lib.or_get_threads.restype = ctypes.c_int
        lib.or_has_openmp.restype = ctypes.c_int
        lib.or_set_threads(default_threads())
        _lib = lib
    return _lib


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _check_state(psi, n):
    if psi.dtype != np.complex128 or not psi.flags.c_contiguous or psi.size != (1 << n):
        raise ValueError("oracle state must be a C-contiguous complex128 array of 2^n entries")


def gate_matrix(name: str, params=(0.0, 0.0, 0.0)) -> np.ndarray:
    """The oracle's 2^k x 2^k matrix for a named gate (first operand most significant)."""
    lib = _load()
    p = np.zeros(3)
    p[:len(params)] = params
    out = np.zeros(16, dtype=np.complex128)
    k = lib.or_gate_matrix(GATE_IDS[name], _dp(p), _dp(out))
    if k < 0:
        raise ValueError(f"unknown gate {name}")
    d = 1 << k
    return out[:d * d].reshape(d, d).copy()


def zero_state(n: int) -> np.ndarray:
    psi = np.zeros(1 << n, dtype=np.complex128)
    psi[0] = 1.0
    return psi


def apply_matrix(psi: np.ndarray, n: int, qubits, u: np.ndarray) -> None:
    """In place: apply the 2^k x 2^k matrix ``u`` on ``qubits`` (Eq. 2 / Eq. 3 form)."""
    _check_state(psi, n)
    lib = _load()
    q = (ctypes.c_int * len(qubits))(*qubits)
    u = np.ascontiguousarray(u, dtype=np.complex128)
    rc = lib.or_apply_matrix(_dp(psi), n, len(qubits), q, _dp(u))
    if rc != 0:
        raise ValueError(f"or_apply_matrix failed ({rc})")


def _marshal(gates):
    ng = len(gates)
    types = np.zeros(ng, dtype=np.int32)
    nq = np.zeros(ng, dtype=np.int32)
    q = np.zeros(ng * 8, dtype=np.int32)
    p = np.zeros(ng * 3, dtype=np.float64)
    dense_off = np.zeros(ng, dtype=np.int64)
    dense_parts = []
    off = 0
    for g, gate in enumerate(gates):
        name, qubits, params = gate
        types[g] = GATE_IDS[name]
        nq[g] = len(qubits)
        q[g * 8:g * 8 + len(qubits)] = qubits
        if name == "dense":
            m = np.ascontiguousarray(params, dtype=np.complex128).reshape(-1)
            dense_off[g] = off
            dense_parts.append(m.view(np.float64))
            off += m.size * 2
        else:
            p[g * 3:g * 3 + len(params)] = params
    dense = np.concatenate(dense_parts) if dense_parts else np.zeros(2)
    return ng, types, nq, q, p, dense, dense_off


def run(psi: np.ndarray, n: int, gates) -> np.ndarray:
    """In place: apply ``gates`` to ``psi`` one by one, in order.  Returns psi."""
    _check_state(psi, n)
    lib = _load()
    ng, types, nq, q, p, dense, dense_off = _marshal(gates)
    ip = ctypes.POINTER(ctypes.c_int)
    rc = lib.or_run(_dp(psi), n, ng, types.ctypes.data_as(ip), nq.ctypes.data_as(ip),
                    q.ctypes.data_as(ip), _dp(p), _dp(dense),
                    dense_off.ctypes.data_as(ctypes.POINTER(ctypes.c_long)))
    if rc != 0:
        raise ValueError(f"oracle rejected gate {-rc - 1}: {gates[-rc - 1]}")
    return psi


def norm(psi: np.ndarray, n: int) -> float:
    """Squared norm sum |a_x|^2 (pairwise summation)."""
    _check_state(psi, n)
    return float(_load().or_norm(_dp(psi), n))


def expz(psi: np.ndarray, n: int) -> np.ndarray:
    """<Z_i> for every qubit i, not divided by the norm."""
    _check_state(psi, n)
    out = np.zeros(n)
    _load().or_expz(_dp(psi), n, _dp(out))
    return out


def top_k(psi: np.ndarray, n: int, k: int):
    """(indices, amplitudes) of the k largest |a|^2, ties to the lower index."""
    _check_state(psi, n)
    idx = np.zeros(k, dtype=np.uint64)
    amp = np.zeros(k, dtype=np.complex128)
    rc = _load().or_top_k(_dp(psi), n, k,
                          idx.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)), _dp(amp))
    if rc != 0:
        raise ValueError("or_top_k failed")
    return idx, amp
