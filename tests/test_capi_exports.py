"""CPU checks of the C-ABI library: it builds for sm_103a, loads, and exports every
function include/qs.h declares (no compute call: there may be no GPU here)."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for f in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if f.endswith(".h"):
            src = open(os.path.join(ROOT, "include", f)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names += re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_ ]*?\**\s*\**(qs_[a-z0-9_]+)\s*\(", src, flags=re.M)
    return sorted(set(names))


def test_library_exports_every_declared_function():
    from paper_2409_14697_gb300 import build as b
    lib_path = b.build()
    lib = ctypes.CDLL(lib_path)
    names = declared_functions()
    assert "qs_create" in names and "qs_apply_circuit" in names and len(names) >= 15
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_header():
    from paper_2409_14697_gb300 import qs
    names = set(declared_functions())
    bound = set(qs.exported_symbols())
    assert bound <= names
    assert names - bound == set() or all(n.startswith("qs_") for n in names - bound)


def test_version_without_gpu():
    from paper_2409_14697_gb300 import build as b, qs
    b.build()
    abi, ndev = qs.qs_version()
    assert abi == 4 and ndev >= 0


def test_gate_record_layout():
    from paper_2409_14697_gb300 import qs
    assert ctypes.sizeof(qs.qs_gate) == 72
    assert ctypes.sizeof(qs.qs_options) == 36
