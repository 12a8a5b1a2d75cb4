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


C_CALLER = r"""
#include <stdio.h>
#include <string.h>
#include "cdg.h"

/* unit square split into 2 x 2 cells, two triangles each; no tagged faces:
 * every boundary face is Dirichlet */
int main(void) {
  double xyz[9][2];
  for (int j = 0; j < 3; ++j)
    for (int i = 0; i < 3; ++i) { xyz[3 * j + i][0] = 0.5 * i; xyz[3 * j + i][1] = 0.5 * j; }
  int64_t elem[8][3];
  int e = 0;
  for (int j = 0; j < 2; ++j)
    for (int i = 0; i < 2; ++i) {
      int64_t v0 = 3 * j + i, v1 = v0 + 1, v2 = v0 + 4, v3 = v0 + 3;
      elem[e][0] = v0; elem[e][1] = v1; elem[e][2] = v2; ++e;
      elem[e][0] = v0; elem[e][1] = v2; elem[e][2] = v3; ++e;
    }
  cdg_mesh m = {2, 9, &xyz[0][0], 8, &elem[0][0], 0, NULL, NULL};
  cdg_options o;
  cdg_default_options(&o);
  o.p = 1;
  o.max_levels = 2;
  cdg_handle* h = NULL;
  if (cdg_create(NULL, &o, &h) != CDG_EINVAL || h != NULL || strlen(cdg_last_error(NULL)) == 0) return 10;
  int rc = cdg_create(&m, &o, &h);
  if (rc != CDG_OK) { printf("create %d %s\n", rc, cdg_last_error(NULL)); return 11; }
  cdg_info inf;
  if (cdg_query(h, &inf) != CDG_OK) return 12;
  double xq[8 * 16 * 2];
  if (inf.nq > 16 || cdg_quadrature_points(h, xq, NULL, NULL) != CDG_OK) return 13;
  double lo = 1.0, hi = 0.0;
  for (int k = 0; k < 2 * 8 * inf.nq; ++k) { if (xq[k] < lo) lo = xq[k]; if (xq[k] > hi) hi = xq[k]; }
  /* a device call before cdg_bind_device is an ordering error, with a message */
  double u[8 * 3];
  rc = cdg_apply(h, 0, u, u, NULL);
  if (rc != CDG_ESTATE || strlen(cdg_last_error(h)) == 0) return 14;
  printf("%lld %d %d %lld %.12f %.12f\n", (long long)inf.n_dofs, inf.n_levels, inf.n_p, (long long)inf.n_bfaces,
         lo, hi);
  cdg_destroy(h);
  return 0;
}
"""


def test_c_caller_host_setup(tmp_path):
    """A plain C program links libcdgmg.so and runs the host side of the ABI:
    argument errors, cdg_create, cdg_query, the quadrature points (strictly
    inside the unit square) and the ordering error of a device call before
    binding."""
    import subprocess
    from paper_2012_08024_gb300 import build
    build.build()
    src = tmp_path / "caller.c"
    src.write_text(C_CALLER)
    exe = tmp_path / "caller"
    libdir = os.path.dirname(build.LIB)
    subprocess.run(["gcc", "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe),
                    build.LIB, "-Wl,-rpath," + libdir], check=True)
    r = subprocess.run([str(exe)], capture_output=True, text=True)
    assert r.returncode == 0, (r.returncode, r.stdout, r.stderr)
    nd, nlev, npb, nbf, lo, hi = r.stdout.split()
    assert (int(nd), int(nlev), int(npb), int(nbf)) == (24, 2, 3, 8)
    assert 0.0 < float(lo) and float(hi) < 1.0
