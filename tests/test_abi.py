"""The C ABI library builds for sm_103a, loads, and exports every declared entry point;
the binding's structs match the header; a plain C program builds against the header.

Only test_c_example_solves (marked gpu) makes CUDA calls; the rest runs on
machines without a GPU.
"""
import ctypes
import os
import re

import pytest

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


# (C struct, ctypes class name in the binding, fields)
LAYOUTS = [
    ("sait_csr", "_Csr", ["n", "nnz", "row_ptr", "col", "val"]),
    ("sait_drop", "_Drop", ["kind", "p", "tau"]),
    ("sait_info", "Info", ["iters", "cycles", "reorth_steps", "pad", "rel_resid"]),
    ("sait_stats", "Stats", ["launches", "ms", "calls"]),
    ("sait_batch_info", "BatchInfo", ["nsys", "converged", "max_iters", "graph_replays", "max_rel_resid", "device_loop",
                                       "graph_launches"]),
    ("sait_tune_report", "TuneReport", ["ncand", "chosen", "format", "lanes", "us"]),
    ("sait_batch_tune_report", "BatchTuneReport", ["ncand", "chosen", "tile_rows", "us"]),
    ("sait_param", "_Param", ["m_terms", "pad", "drop"]),
    ("sait_param_report", "ParamReport",
     ["ncand", "chosen", "status", "iters", "nnz", "build_ms", "solve_ms", "rel_resid"]),
]


def test_binding_structs_match_the_header(tmp_path):
    """Every struct the binding passes by pointer has the header's size and
    field offsets (a C program compiled against include/sait.h prints them)."""
    import shutil
    import subprocess
    import paper_2106_12836_gb300 as sg
    cc = shutil.which("gcc") or shutil.which("cc")
    assert cc, "a C compiler is needed to read the header's layouts"
    lines = ['#include <stddef.h>', '#include <stdio.h>', '#include "sait.h"', "int main(void) {"]
    for cname, _, fields in LAYOUTS:
        lines.append(f'  printf("{cname} size %zu\\n", sizeof({cname}));')
        for f in fields:
            lines.append(f'  printf("{cname} {f} %zu\\n", offsetof({cname}, {f}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    c = {}
    for line in out:
        if line:
            name, key, val = line.split()
            c[(name, key)] = int(val)
    for cname, pyname, fields in LAYOUTS:
        cls = getattr(sg, pyname)
        assert ctypes.sizeof(cls) == c[(cname, "size")], cname
        for f in fields:
            assert getattr(cls, f).offset == c[(cname, f)], (cname, f)


def test_binding_fails_loudly_without_the_library(monkeypatch, tmp_path):
    """No CPU fallback: with the library missing, the first call raises."""
    import pytest
    import paper_2106_12836_gb300 as sg
    monkeypatch.setattr(sg, "_lib", None)
    monkeypatch.setattr(sg._build, "LIB", str(tmp_path / "missing" / "libsait.so"))
    with pytest.raises(ImportError):
        sg.sait_status_string(0)


def test_binding_rejects_host_tensors():
    """Vectors must be device tensors: host memory is refused before any call."""
    import pytest
    import torch
    import paper_2106_12836_gb300 as sg
    with pytest.raises(ValueError):
        sg._vec(torch.zeros(4, dtype=torch.float64), 4, "x")
    with pytest.raises(ValueError):
        sg._ptr(torch.zeros(4, dtype=torch.float64))


def _build_c_example(tmp_path):
    import shutil
    import subprocess
    from paper_2106_12836_gb300 import build
    lib = build.build()
    cc = shutil.which("gcc") or shutil.which("cc")
    assert cc, "a C compiler is needed"
    cuda = os.environ.get("CUDA_HOME", "/usr/local/cuda")
    exe = tmp_path / "c_api_example"
    subprocess.run([cc, "-std=c11", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"),
                    "-I", os.path.join(cuda, "include"), os.path.join(ROOT, "tests", "c_api_example.c"),
                    "-L", os.path.dirname(lib), "-lsait", "-L", os.path.join(cuda, "lib64"), "-lcudart", "-lm",
                    "-o", str(exe)], check=True)
    return exe, [os.path.dirname(lib), os.path.join(cuda, "lib64")]


def test_c_example_compiles_against_the_header_and_links(tmp_path):
    """A C program using include/sait.h alone builds and links against libsait.so."""
    exe, _ = _build_c_example(tmp_path)
    assert exe.exists()


@pytest.mark.gpu
def test_c_example_solves(tmp_path):
    """The C program runs the whole path (ILU(0), SAIT build, GMRES) through the
    C ABI and reaches a true relative residual of 1e-8."""
    import subprocess
    exe, libdirs = _build_c_example(tmp_path)
    env = dict(os.environ, LD_LIBRARY_PATH=":".join(libdirs + [os.environ.get("LD_LIBRARY_PATH", "")]))
    r = subprocess.run([str(exe), "48"], capture_output=True, text=True, env=env, timeout=120)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "relative residual" in r.stdout
