"""Builds tests/ix_check.cpp (the host build of the integer-product arithmetic of
complex128 streaming updates) with g++; used by the CPU and GPU tests of that arithmetic."""
import shutil
import subprocess
from pathlib import Path

import pytest

ROOT = Path(__file__).resolve().parents[1]
CSRC = ROOT / "paper_2409_14697_gb300" / "csrc"


def build_ix_check(out_dir: Path) -> Path:
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ is not available")
    exe = out_dir / "ix_check"
    cmd = [gxx, "-O2", "-std=c++17", f"-I{CSRC}", str(ROOT / "tests" / "ix_check.cpp"), "-o", str(exe)]
    r = subprocess.run(cmd, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-4000:]
    return exe
