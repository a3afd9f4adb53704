"""CPU test of the host rewrites the executor applies before its kernels run (global-phase
fold, deferred Hadamard scale, gate fusion, U3 split, diagonal merge with non-local
controlled phases, their chunk-pass order, the Tensor Product Booster's prefix and groups,
and the complex64 register-phase programs, interpreted thread by thread as the chunk
kernel runs them): builds ``host_transforms_check.cpp``
against the package's host sources with g++ and runs it on seeded random circuits.  Each
rewrite must leave a 10-qubit state unchanged to 1e-12 and keep the limits the kernels
rely on; the resulting tile programs (kernel ops on tile positions, with non-local terms
and Hadamards joined with their controlled blocks) are interpreted tile by tile and must
give the same state.  The whole planned complex128 path is emulated too: the planner and
per-pass programs as the library runs them (merged diagonal runs applied from their
documented table semantics), every op exactly once, the same final state.  No GPU: the
CUDA headers and runtime library are needed only to link; every launcher is a stub that
fails."""
import os
import shutil
import subprocess
from pathlib import Path

import numpy as np
import pytest

import oracle
from paper_2409_14697_gb300 import qs

ROOT = Path(__file__).resolve().parents[1]
CSRC = ROOT / "paper_2409_14697_gb300" / "csrc"


def _cuda_include():
    for base in (os.environ.get("CUDA_HOME"), os.environ.get("CUDA_PATH"), "/usr/local/cuda"):
        if base and (Path(base) / "include" / "cuda_runtime.h").exists():
            return str(Path(base) / "include")
    nvcc = shutil.which("nvcc")
    if nvcc:
        inc = Path(nvcc).resolve().parents[1] / "include"
        if (inc / "cuda_runtime.h").exists():
            return str(inc)
    return None


@pytest.fixture(scope="module")
def checker(tmp_path_factory):
    gxx = shutil.which("g++")
    inc = _cuda_include()
    if gxx is None or inc is None:
        pytest.skip("g++ or the CUDA headers are not available")
    # the planner's host code references the CUDA runtime (never called here)
    lib = Path(inc).parent / "lib64"
    if not any(lib.glob("libcudart.so*")):
        pytest.skip("the CUDA runtime library is not available")
    exe = tmp_path_factory.mktemp("host_transforms") / "host_transforms_check"
    srcs = [ROOT / "tests" / "host_transforms_check.cpp"] + \
        [CSRC / f for f in ("ir.cpp", "kgeom.cpp", "plan.cpp", "phasefn.cpp", "tpb.cpp")]
    cmd = [gxx, "-O1", "-std=c++17", f"-I{CSRC}", f"-I{ROOT / 'include'}", f"-I{inc}",
           *map(str, srcs), f"-L{lib}", "-lcudart", f"-Wl,-rpath,{lib}", "-o", str(exe)]
    r = subprocess.run(cmd, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-4000:]
    return exe


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_host_rewrites_keep_the_circuit(checker, seed):
    r = subprocess.run([str(checker), str(seed), "24"], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0 and "OK" in r.stdout, r.stdout[-4000:]


def test_lowered_gates_equal_the_oracle_matrices(checker):
    """Every fixed gate type as the library lowers it (the matrices all of the checks above
    start from) equals the oracle's matrix for that gate, at several angle sets."""
    r = subprocess.run([str(checker), "--gates"], capture_output=True, text=True, timeout=60)
    assert r.returncode == 0, r.stderr[-2000:]
    names = {v: k for k, v in qs.GATE_TYPES.items()}
    lines = r.stdout.strip().splitlines()
    assert len(lines) == 17 * 4
    for line in lines:
        f = line.split()
        name, params, k = names[int(f[0])], tuple(float(x) for x in f[1:4]), int(f[4])
        vals = np.array([float(x) for x in f[5:]])
        got = (vals[0::2] + 1j * vals[1::2]).reshape(1 << k, 1 << k)
        want = oracle.gate_matrix(name, params)
        assert got.shape == want.shape, name
        assert np.max(np.abs(got - want)) <= 1e-15, (name, params)
