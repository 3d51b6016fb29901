"""The C-ABI library builds for sm_103a, loads without a GPU and exports
every symbol that include/ctbop.h declares; the binding's structs have the
C layout."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "ctbop.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(ctbop_[a-z_0-9]+)\s*\(", src)))


def test_library_builds_and_exports_declared_symbols():
    from paper_1802_07871_gb300 import build, ctbop
    path = build.build()
    lib = ctypes.CDLL(path)
    names = _declared()
    assert len(names) >= 17
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) == set(ctbop.EXPORTS)


def test_struct_layouts_match_header(tmp_path):
    from paper_1802_07871_gb300 import ctbop
    c = tmp_path / "sz.c"
    c.write_text('#include <stdio.h>\n#include "ctbop.h"\nint main(){printf("%zu %zu %zu %zu\\n",'
                 'sizeof(ctbop_params), sizeof(ctbop_options), sizeof(ctbop_stats), sizeof(ctbop_peaks));}\n')
    exe = tmp_path / "sz"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(c), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()
    assert [int(v) for v in out] == [ctypes.sizeof(ctbop.Params), ctypes.sizeof(ctbop.Options),
                                     ctypes.sizeof(ctbop.Stats), ctypes.sizeof(ctbop.Peaks)]


def test_params_marshalling_l1_padding():
    from paper_1802_07871_gb300 import ctbop, structures as st
    p = ctbop.params_struct(st.load_params("pt"))
    assert p.g[1][1] == 1e30 and p.gamma[3][1] == 0.0
    p1 = ctbop.params_struct(st.load_params("p1"))
    assert p1.g[2][0] != p1.g[1][0]   # ordered pairs kept apart
