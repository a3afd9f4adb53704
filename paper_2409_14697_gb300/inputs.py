"""Seeded synthetic inputs: circuits (gate lists) and initial states.

This module holds no simulation arithmetic.  It only draws angles, graphs and
Gaussian numbers, so that the CUDA path and the CPU oracle can be fed the same
inputs.  A gate is a tuple ``(name, qubits, params)`` with ``name`` one of
``h x y z s t rx ry rz p u3 cnot cz swap cu3 cp rzz``, or
``("dense", qubits, matrix)``.  For multi-qubit gates the first operand is the
most significant bit of the gate's group index, the row order of Eq. 3 of
QueenV2 (arXiv 2409.14697), so ``cnot`` and ``cu3`` take (control, target).

Workload families (readings of unspecified details are fixed here):
  * ``brickwork``: per layer, U3 with angles U[0, 2pi) on every qubit, then CZ on
    pairs (0,1),(2,3),... on even layers and (1,2),(3,4),... on odd layers (open
    chain, no wrap-around).
  * ``gate_sweep``: one gate type applied across targets 0..n-1; two-qubit gates on
    (q, q+1 mod n).
  * ``qaoa_3regular``: H on all, then p layers of [RZZ(gamma) on every edge,
    RX(beta) on every qubit], gamma, beta ~ U[0, pi), on a seeded 3-regular graph
    (for odd n: a 3-regular graph on n-1 vertices with one edge (u,v) replaced by
    (u,n-1),(v,n-1)).
  * ``qaoa_complete``: the same on the complete graph (QueenV2 Table IV family).
  * ``tfim``: first-order Trotter steps of H = -J sum Z_i Z_{i+1} - h sum X_i (open
    chain): RZZ(-2 J dt) on every bond, then RX(-2 h dt) on every qubit.
  * ``qft``: H and controlled phases CP(pi / 2^d), then the final qubit reversal
    by SWAPs (QueenV2 Table III family).
"""
from __future__ import annotations

import math

import numpy as np

MASTER_SEED = 20240922

SWEEP_GATES = ("h", "x", "rz", "u3", "cnot", "cz", "swap", "cu3")

_ARITY = {"h": 1, "x": 1, "y": 1, "z": 1, "s": 1, "t": 1, "rx": 1, "ry": 1,
          "rz": 1, "p": 1, "u3": 1, "cnot": 2, "cz": 2, "swap": 2, "cu3": 2,
          "cp": 2, "rzz": 2}
_NPARAM = {"rx": 1, "ry": 1, "rz": 1, "p": 1, "u3": 3, "cu3": 3, "cp": 1, "rzz": 1}


def arity(name: str) -> int:
    return _ARITY[name]


def n_params(name: str) -> int:
    return _NPARAM.get(name, 0)


def rng(*key: int) -> np.random.Generator:
    """A numpy generator seeded by (MASTER_SEED, *key)."""
    return np.random.default_rng(np.random.SeedSequence([MASTER_SEED, *[int(k) for k in key]]))


def brickwork(n: int, layers: int, seed: int = 1):
    """Random U3 + CZ brickwork circuit (angles drawn per layer, qubit, (theta, phi, lambda))."""
    r = rng(1, seed, n, layers)
    gates = []
    for layer in range(layers):
        ang = r.uniform(0.0, 2.0 * math.pi, size=(n, 3))
        for q in range(n):
            gates.append(("u3", (q,), tuple(float(a) for a in ang[q])))
        for a in range(layer % 2, n - 1, 2):
            gates.append(("cz", (a, a + 1), ()))
    return gates


def gate_sweep(n: int, name: str, seed: int = 2, count: int | None = None):
    """``count`` (default n) applications of one gate type on targets q = 0, 1, ... (mod n)."""
    r = rng(2, seed, n, list(_ARITY).index(name))
    count = n if count is None else count
    gates = []
    for i in range(count):
        q = i % n
        qubits = (q,) if _ARITY[name] == 1 else (q, (q + 1) % n)
        params = tuple(float(a) for a in r.uniform(0.0, 2.0 * math.pi, size=n_params(name)))
        gates.append((name, qubits, params))
    return gates


def sweep_all(n: int, seed: int = 2, count: int | None = None):
    """The 30-qubit gate-benchmark sequence: every type of SWEEP_GATES, one after another."""
    out = []
    for name in SWEEP_GATES:
        out.extend(gate_sweep(n, name, seed, count))
    return out


def random_3regular(n: int, seed: int = 3):
    """Edges of a seeded random 3-regular (multi-edge and loop free) graph on n vertices.

    Pairing model with rejection.  For odd n see the module docstring."""
    r = rng(3, seed, n)
    m = n if n % 2 == 0 else n - 1
    if m < 4:
        raise ValueError("need at least 4 vertices")
    while True:
        stubs = np.repeat(np.arange(m), 3)
        r.shuffle(stubs)
        pairs = stubs.reshape(-1, 2)
        if np.any(pairs[:, 0] == pairs[:, 1]):
            continue
        e = {tuple(sorted((int(a), int(b)))) for a, b in pairs}
        if len(e) == len(pairs):
            break
    edges = sorted(e)
    if n != m:
        k = int(r.integers(len(edges)))
        u, v = edges.pop(k)
        edges += [(u, n - 1), (v, n - 1)]
    return edges


def _qaoa(n, edges, p, r):
    gates = [("h", (q,), ()) for q in range(n)]
    for _ in range(p):
        gamma, beta = r.uniform(0.0, math.pi, size=2)
        gates += [("rzz", (a, b), (float(gamma),)) for a, b in edges]
        gates += [("rx", (q,), (float(beta),)) for q in range(n)]
    return gates


def qaoa_3regular(n: int, p: int = 4, seed: int = 3):
    """QAOA MaxCut circuit on a seeded 3-regular graph, p layers."""
    return _qaoa(n, random_3regular(n, seed), p, rng(4, seed, n, p))


def qaoa_complete(n: int, p: int = 5, seed: int = 5):
    """QAOA on the complete graph, p layers (the fully connected benchmark family)."""
    edges = [(a, b) for a in range(n) for b in range(a + 1, n)]
    return _qaoa(n, edges, p, rng(5, seed, n, p))


def tfim(n: int, steps: int = 50, dt: float = 0.05, J: float = 1.0, h: float = 1.0):
    """First-order Trotter circuit of the open transverse-field Ising chain."""
    gates = []
    for _ in range(steps):
        gates += [("rzz", (q, q + 1), (-2.0 * J * dt,)) for q in range(n - 1)]
        gates += [("rx", (q,), (-2.0 * h * dt,)) for q in range(n)]
    return gates


def qft(n: int):
    """Textbook QFT on n qubits: H on qubit j then CP(pi/2^d) from lower qubits, top qubit first."""
    gates = []
    for j in reversed(range(n)):
        gates.append(("h", (j,), ()))
        for d, k in enumerate(reversed(range(j)), start=1):
            gates.append(("cp", (k, j), (math.pi / 2 ** d,)))
    for a in range(n // 2):
        gates.append(("swap", (a, n - 1 - a), ()))
    return gates


def inverse(gates):
    """The inverse circuit: reversed order, each gate replaced by its inverse."""
    out = []
    for name, qubits, params in reversed(gates):
        if name in ("h", "x", "y", "z", "cnot", "cz", "swap"):
            out.append((name, qubits, params))
        elif name in ("rx", "ry", "rz", "p", "cp", "rzz"):
            out.append((name, qubits, (-params[0],)))
        elif name in ("u3", "cu3"):
            t, ph, la = params
            out.append((name, qubits, (-t, -la, -ph)))
        elif name == "s":
            out.append(("p", qubits, (-math.pi / 2,)))
        elif name == "t":
            out.append(("p", qubits, (-math.pi / 4,)))
        elif name == "dense":
            out.append(("dense", qubits, np.conj(np.asarray(params)).T.copy()))
        else:
            raise ValueError(name)
    return out


def gaussian_state(n: int, seed: int = 7, dtype=np.complex128, out: np.ndarray | None = None) -> np.ndarray:
    """i.i.d. N(0,1) real and imaginary parts, scaled to unit norm (sum of squares in FP64).

    ``out`` (a C-contiguous complex array of 2^n entries, e.g. pinned host memory) is
    filled in place when given; its dtype wins over ``dtype``."""
    r = rng(7, seed, n)
    psi = np.empty(1 << n, dtype=dtype) if out is None else out
    v = psi.view(np.float64 if psi.dtype == np.complex128 else np.float32)
    chunk = 1 << 24
    s = 0.0
    for lo in range(0, v.size, chunk):
        x = r.standard_normal(min(chunk, v.size - lo))
        v[lo:lo + chunk] = x
        s += float(np.dot(x, x))
    scale = 1.0 / math.sqrt(s)
    for lo in range(0, v.size, chunk):
        v[lo:lo + chunk] *= scale
    return psi


def random_circuit(n: int, ng: int, seed: int = 8, names=None):
    """ng random gates of mixed types on random distinct qubits (for exhaustive tests)."""
    r = rng(8, seed, n, ng)
    names = names or [g for g in _ARITY if _ARITY[g] <= n]
    gates = []
    for _ in range(ng):
        name = names[int(r.integers(len(names)))]
        qubits = tuple(int(x) for x in r.choice(n, size=_ARITY[name], replace=False))
        params = tuple(float(a) for a in r.uniform(0.0, 2.0 * math.pi, size=n_params(name)))
        gates.append((name, qubits, params))
    return gates


def random_unitary(k: int, seed: int = 9) -> np.ndarray:
    """Haar-like random 2^k x 2^k unitary (QR of a complex Gaussian matrix)."""
    r = rng(9, seed, k)
    d = 1 << k
    z = (r.standard_normal((d, d)) + 1j * r.standard_normal((d, d))) / math.sqrt(2.0)
    qm, rm = np.linalg.qr(z)
    return qm * (np.diag(rm) / np.abs(np.diag(rm)))


def batched_circuits(count: int = 4096, seed: int = 10, n_range=(8, 20), depth_range=(10, 60)):
    """(n, gates) pairs: n ~ U{n_lo..n_hi}, depth ~ U{d_lo..d_hi} brickwork layers."""
    r = rng(10, seed, count)
    out = []
    for i in range(count):
        n = int(r.integers(n_range[0], n_range[1] + 1))
        d = int(r.integers(depth_range[0], depth_range[1] + 1))
        out.append((n, brickwork(n, d, seed=1000 * seed + i)))
    return out


def served_stream(count: int, rate_hz: float = 2000.0, seed: int = 11, n_range=(10, 30)):
    """Poisson request stream: list of dicts (t_arrival, n, dtype, family, gates, init_seed).

    n is log-uniform on [n_lo, n_hi]; family is 'brickwork' (20 layers from |0>) or
    'sweep' (30 applications of one random gate type on a Gaussian state); dtype is
    complex64 or complex128 with equal probability."""
    r = rng(11, seed, count)
    t = 0.0
    reqs = []
    for i in range(count):
        t += float(r.exponential(1.0 / rate_hz))
        n = int(math.floor(math.exp(r.uniform(math.log(n_range[0]), math.log(n_range[1] + 1)))))
        n = min(max(n, n_range[0]), n_range[1])
        fam = "brickwork" if r.random() < 0.5 else "sweep"
        dt = "c64" if r.random() < 0.5 else "c128"
        if fam == "brickwork":
            gates = brickwork(n, 20, seed=50000 + i)
        else:
            gname = SWEEP_GATES[int(r.integers(len(SWEEP_GATES)))]
            gates = gate_sweep(n, gname, seed=60000 + i, count=30)
        reqs.append({"t": t, "n": n, "dtype": dt, "family": fam, "gates": gates,
                     "init_seed": 70000 + i if fam == "sweep" else None})
    return reqs
