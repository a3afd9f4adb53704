"""CPU test of the integer-product arithmetic of complex128 streaming updates
(``csrc/ixmath.cuh``, QS_PREC_IX64), built for the host with g++ from the same header the
kernels include.  ``ix_check`` draws seeded one-qubit updates (U3-class, general unitary
and diagonal factors, Eq. 2) on amplitudes of several magnitude profiles and checks each
real output against the exact sum in binary128: within 0.5 ulp + 2^-56.4 of the largest
|matrix entry x amplitude|, both result encodings bitwise equal, and the largest error no
larger than that of the native FP64 multiply-add chains of the FP64 kernels."""
import subprocess

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
