"""Full-size GPU parity against the FP64 oracle, through the C ABI.

The oracle runs on every host core (its threads give results bitwise equal to one
thread), so it finishes the benchmark sizes in minutes.

* The 30-qubit gate benchmark: a seeded Gaussian state; H, X, RZ, U3, CNOT, CZ, SWAP and
  CU3 each applied 30 times across the targets (two-qubit gates on (q, q+1 mod 30)).
  After each type the GPU states are compared element by element with the oracle's:
  complex128 gate by gate (native FP64, integer-product and double-float arithmetic) and as
  one planned call
  per type (max-abs <= 1e-12), complex64 gate by gate and planned (1 - F <= 1e-6 and the
  max-abs bound of the complex64 tests).
* The same sweep at 22 qubits, where every streaming kernel instance runs grids of several
  iterations per CTA.
* The three circuit families of the 33-qubit benchmark at 28 qubits (brickwork of 40 U3+CZ
  layers, QAOA p=4 on a 3-regular graph, TFIM 50 Trotter steps), complex64 with register
  phases and with tensor-core blocks, against the complex128 oracle from |0...0>.
* At 33 qubits (64 GiB complex64), where no oracle state fits the host comfortably:
  norm, inverse-circuit fidelity, and for QAOA the bit-flip symmetry a_x = a_~x and
  <Z_q> = 0 that hold exactly for H^n|0> followed by RZZ and RX layers.
"""
import time

import numpy as np
import pytest

import oracle
from paper_2409_14697_gb300 import inputs
from tests.gpu_util import TOL_C128, TOL_C64, compare_large, require_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def qs():
    require_gpu()
    from paper_2409_14697_gb300 import qs as q
    q.load()
    return q


def _pinned(nbytes):
    torch = pytest.importorskip("torch")
    return torch.empty(nbytes, dtype=torch.uint8, pin_memory=True)


def _download(qs, h, n, buf, npdt):
    """State -> pinned host buffer (copy kernel over the CPU-GPU link); a numpy view."""
    qs.qs_amplitudes_into(h, 0, 1 << n, buf.data_ptr())
    return buf.numpy()[:np.dtype(npdt).itemsize << n].view(npdt)


def _sweep_parity(qs, n, c64_planned=True):
    """Gate benchmark of every SWEEP_GATES type at n qubits; compares after each type.
    Returns a dict of per-type errors and timings (printed with -s)."""
    psi = inputs.gaussian_state(n, seed=2024)
    variants = [("c128_gate", 2, qs.QS_MODE_GATE, qs.QS_PREC_FP64),
                ("c128_ix64_gate", 2, qs.QS_MODE_GATE, qs.QS_PREC_IX64),
                ("c128_planned", 2, qs.QS_MODE_AUTO, qs.QS_PREC_FP64),
                ("c128_planned_ix64", 2, qs.QS_MODE_AUTO, qs.QS_PREC_IX64),
                ("c128_df32_gate", 2, qs.QS_MODE_GATE, qs.QS_PREC_DF32),
                ("c64_gate", 1, qs.QS_MODE_GATE, 0)]
    if c64_planned:
        variants.append(("c64_planned", 1, qs.QS_MODE_AUTO, 0))
    hs = {}
    report = {"oracle_threads": oracle.threads(), "types": {}}
    try:
        for name, dt, _, _ in variants:
            hs[name] = qs.qs_create(n, dt)
            qs.qs_set_amplitudes(hs[name], psi if dt == 2 else psi.astype(np.complex64))
        buf = _pinned(16 << n)
        t_or = 0.0
        for gname in inputs.SWEEP_GATES:
            seg = inputs.gate_sweep(n, gname, seed=2, count=n)
            for name, dt, mode, prec in variants:
                qs.qs_apply_circuit(hs[name], seg, qs.options(mode=mode, precision=prec))
            t0 = time.time()
            oracle.run(psi, n, seg)
            t_or += time.time() - t0
            row = {}
            for name, dt, mode, prec in variants:
                got = _download(qs, hs[name], n, buf, np.complex128 if dt == 2 else np.complex64)
                err, gap = compare_large(got, psi)
                row[name] = (err, gap)
                if dt == 2:
                    assert err <= TOL_C128, (gname, name, err)
                else:
                    assert err <= TOL_C64, (gname, name, err)
                    assert gap <= 1e-6, (gname, name, gap)
            report["types"][gname] = row
        report["oracle_s"] = t_or
    finally:
        for h in hs.values():
            qs.qs_destroy(h)
    print(report)
    return report


def test_gate_benchmark_30q_every_type_vs_oracle(qs):
    """The headline workload at full size: 2^30 amplitudes, all 240 gates."""
    _sweep_parity(qs, 30)


def test_gate_benchmark_22q_every_type_vs_oracle(qs):
    """22 qubits: the streaming kernels' persistent grids loop several times per CTA."""
    _sweep_parity(qs, 22)


FAMILIES = {
    "brickwork40": lambda n: inputs.brickwork(n, 40, seed=3),
    "qaoa_p4": lambda n: inputs.qaoa_3regular(n, p=4, seed=3),
    "tfim50": lambda n: inputs.tfim(n, steps=50, dt=0.05),
}


@pytest.mark.parametrize("family", list(FAMILIES))
def test_circuit_families_28q_vs_oracle(qs, family):
    """Each 33-qubit benchmark family at 28 qubits, complex64, register phases and
    tensor-core blocks (fusion width 5), element by element against the oracle."""
    n = 28
    gates = FAMILIES[family](n)
    t0 = time.time()
    want = oracle.run(oracle.zero_state(n), n, gates)
    t_or = time.time() - t0
    buf = _pinned(8 << n)
    out = {}
    for label, fk in (("register_phases", 0), ("tensor_cores", 5)):
        h = qs.qs_create(n, 1)
        try:
            qs.qs_apply_circuit(h, gates, qs.options(fuse_k=fk))
            st = qs.qs_last_stats(h)
            got = _download(qs, h, n, buf, np.complex64)
            err, gap = compare_large(got, want)
        finally:
            qs.qs_destroy(h)
        out[label] = (err, gap, st["passes"], st["tc_blocks"])
        assert err <= TOL_C64, (label, err)
        assert gap <= 1e-6, (label, gap)
        if fk:
            assert st["tc_blocks"] > 0
        else:
            assert st["tc_blocks"] == 0
    print({"family": family, "gates": len(gates), "oracle_s": t_or, **out})


@pytest.mark.parametrize("family", list(FAMILIES))
def test_circuit_families_33q_norm_inverse_symmetry(qs, family):
    """33 qubits complex64 (64 GiB): the circuit keeps the norm; the circuit followed by
    its inverse returns |0...0>; QAOA keeps a_x = a_~x and <Z_q> = 0."""
    n = 33
    gates = FAMILIES[family](n)
    h = qs.qs_create(n, 1)
    try:
        qs.qs_apply_circuit(h, gates)
        ez, nrm = qs.qs_expectation_z(h)
        assert abs(nrm - 1.0) <= 1e-4, nrm
        if family == "qaoa_p4":
            assert np.max(np.abs(ez)) <= 1e-5, np.max(np.abs(ez))
            w = 1 << 12
            lo = qs.qs_amplitudes(h, 0, w).astype(np.complex128)
            hi = qs.qs_amplitudes(h, (1 << n) - w, w).astype(np.complex128)[::-1]
            # x and ~x = 2^n - 1 - x: the low block against the reversed high block
            assert np.max(np.abs(lo - hi)) <= 1e-4 * np.max(np.abs(lo)), np.max(np.abs(lo - hi))
        qs.qs_apply_circuit(h, inputs.inverse(gates))
        a0 = qs.qs_amplitudes(h, 0, 1).astype(np.complex128)[0]
        nrm2 = qs.qs_norm(h)
        gap = 1.0 - abs(a0) ** 2 / nrm2
        assert gap <= 1e-6, gap
        print({"family": family, "norm_after": nrm, "inverse_1mF": gap})
    finally:
        qs.qs_destroy(h)
