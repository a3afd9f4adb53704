"""CPU test of the integer-product arithmetic of complex128 streaming updates
(``csrc/ixmath.cuh``, QS_PREC_IX64), built for the host with g++ from the same header the
kernels include.  ``ix_check`` draws seeded one-qubit updates (U3-class, general unitary
and diagonal factors, Eq. 2) on amplitudes of several magnitude profiles and checks each
real output against the exact sum in binary128: within 0.5 ulp + 2^-56.4 of the largest
|matrix entry x amplitude|, both result encodings bitwise equal, and the largest error no
larger than that of the native FP64 multiply-add chains of the FP64 kernels.  Its
``--apply`` mode (the reference the GPU bit-for-bit test uses) is checked against the
oracle's dense application of each form's matrices."""
import subprocess

import numpy as np
import pytest

from tests.ix_build import build_ix_check


@pytest.fixture(scope="module")
def ix_check(tmp_path_factory):
    return build_ix_check(tmp_path_factory.mktemp("ix"))


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_integer_products_within_bound_of_exact(ix_check, seed):
    r = subprocess.run([str(ix_check), str(seed), "300000"], capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stdout[-4000:]
    assert r.stdout.strip().endswith("OK")
    stats = r.stdout.split()
    # the integer form's worst error is at most native FP64's, in units of the largest term
    ix_err = float(stats[stats.index("max_err_ix") + 1])
    nat_err = float(stats[stats.index("max_err_native") + 1])
    assert ix_err <= nat_err


FORMS = {
    # (form, matrix builder): the 2x2 matrices the library routes to each integer form
    "r0": lambda r: _real_first(r),
    "gen": lambda r: _unitary(r),
    "real": lambda r: _rot(r.uniform(0, 2 * np.pi)),
    "rx": lambda r: _rx(r.uniform(0, 2 * np.pi)),
}


def _unitary(r):
    z = r.standard_normal((2, 2)) + 1j * r.standard_normal((2, 2))
    q, rr = np.linalg.qr(z)
    return q * (np.diag(rr) / np.abs(np.diag(rr)))


def _real_first(r):
    u = _unitary(r)
    u = u * np.exp(-1j * np.angle(u[0, 0]))
    u[0, 0] = abs(u[0, 0])
    return u


def _rot(a):
    return np.array([[np.cos(a), -np.sin(a)], [np.sin(a), np.cos(a)]], dtype=np.complex128)


def _rx(a):
    return np.array([[np.cos(a), -1j * np.sin(a)], [-1j * np.sin(a), np.cos(a)]])


@pytest.mark.parametrize("form", list(FORMS) + ["phase"])
@pytest.mark.parametrize("q", [0, 4, 9])
def test_apply_matches_the_oracle(ix_check, tmp_path, form, q):
    """One gate on a 10-qubit state through the host build of the integer form (every pair,
    or every element with bit q set for a phase) against the oracle's dense application:
    within 0.5 ulp + 2^-56.4 of the largest term, far inside 1e-15 of the largest amplitude."""
    import oracle
    from paper_2409_14697_gb300 import inputs
    n = 10
    r = np.random.default_rng(1000 + q)
    psi = inputs.gaussian_state(n, seed=77 + q)
    if form == "phase":
        a = r.uniform(0, 2 * np.pi)
        m = np.array([np.cos(a), np.sin(a)])
        u = np.diag([1.0, np.cos(a) + 1j * np.sin(a)])
    else:
        u = FORMS[form](r)
        m = np.ascontiguousarray(u, dtype=np.complex128).reshape(-1).view(np.float64)
    (tmp_path / "psi.bin").write_bytes(psi.tobytes())
    (tmp_path / "m.bin").write_bytes(np.ascontiguousarray(m, dtype=np.float64).tobytes())
    res = subprocess.run([str(ix_check), "--apply", form, str(n), str(q), str(tmp_path / "psi.bin"),
                          str(tmp_path / "m.bin"), str(tmp_path / "out.bin")], capture_output=True, text=True)
    assert res.returncode == 0, res.stdout
    got = np.frombuffer((tmp_path / "out.bin").read_bytes(), dtype=np.complex128)
    want = psi.copy()
    oracle.apply_matrix(want, n, (q,), u)
    assert np.max(np.abs(got - want)) <= 1e-15 * np.max(np.abs(psi))
