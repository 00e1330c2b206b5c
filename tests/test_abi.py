"""The C ABI library builds for sm_103a, loads, and exports every declared entry point.

No CUDA call is made: this runs on machines without a GPU.
"""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            src = open(os.path.join(ROOT, "include", f)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(sait_\w+)\s*\(", src))
    return names


def test_library_exports_every_declared_symbol():
    from paper_2106_12836_gb300 import build
    lib = ctypes.CDLL(build.build())
    names = declared()
    assert len(names) >= 20
    missing = [n for n in sorted(names) if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_the_abi():
    import paper_2106_12836_gb300 as sg
    assert set(sg.EXPORTS) == declared()
    for n in sg.EXPORTS:
        assert callable(getattr(sg, n))


def test_status_strings_without_gpu():
    import paper_2106_12836_gb300 as sg
    assert sg.sait_status_string(0) == "ok"
    assert "triangular" in sg.sait_status_string(2)
    assert sg.sait_status_string(99) == "unknown status"
