"""The C ABI library loads and exports every function include/cdg.h declares,
with the binding's signature table covering exactly those (no device calls)."""
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared():
    names = []
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", f)).read()
            names += re.findall(r"^\s*(?:int|int64_t|void|const char\*)\s+(cdg_\w+)\s*\(", txt, re.M)
    return names


def test_every_declared_symbol_is_exported():
    from paper_2012_08024_gb300 import build, SIGNATURES
    build.build()
    import ctypes
    L = ctypes.CDLL(build.LIB)
    names = declared()
    assert len(names) >= 20
    for n in names:
        assert hasattr(L, n), n
    assert sorted(names) == sorted(SIGNATURES), set(names) ^ set(SIGNATURES)


def test_binding_loads_library():
    import paper_2012_08024_gb300 as pkg
    L = pkg.lib()
    import ctypes
    o = pkg.cdg_options()
    L.cdg_default_options(ctypes.byref(o))
    assert o.p == 2 and abs(o.omega - 2 / 3) < 1e-15 and o.tol == 1e-10 and o.maxit == 500


def test_struct_layouts_match_the_header(tmp_path):
    """The ctypes mirrors of cdg_mesh, cdg_options and cdg_info have the field
    offsets and sizes that a C compiler gives the header's structs."""
    import ctypes
    import subprocess
    from paper_2012_08024_gb300 import cdg_info, cdg_mesh, cdg_options
    structs = {"cdg_mesh": cdg_mesh, "cdg_options": cdg_options, "cdg_info": cdg_info}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "cdg.h"', 'int main(void) {']
    for sname, cls in structs.items():
        lines.append(f'  printf("{sname} sizeof %zu\\n", sizeof({sname}));')
        for fname, _ in cls._fields_:
            lines.append(f'  printf("{sname} {fname} %zu\\n", offsetof({sname}, {fname}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {tuple(l.split()[:2]): int(l.split()[2]) for l in out if l.strip()}
    for sname, cls in structs.items():
        assert got[(sname, "sizeof")] == ctypes.sizeof(cls), sname
        for fname, _ in cls._fields_:
            assert got[(sname, fname)] == getattr(cls, fname).offset, (sname, fname)


def test_binding_rejects_host_tensors_before_the_library():
    """Device entry points take CUDA tensors only: a host tensor is refused by the
    binding (ValueError) and never reaches a kernel; None stays None (nullable)."""
    import torch
    from paper_2012_08024_gb300 import _dvec
    with pytest.raises(ValueError, match="CUDA tensor"):
        _dvec(torch.zeros(4, dtype=torch.float64), 4, "x")
    with pytest.raises(ValueError, match="CUDA tensor"):
        _dvec(np.zeros(4), 4, "x")
    assert _dvec(None, 4, "gD") is None
