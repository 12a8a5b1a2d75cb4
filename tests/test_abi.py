"""The C ABI library loads and exports every function include/cdg.h declares,
with the binding's signature table covering exactly those (no device calls)."""
import os
import re

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
