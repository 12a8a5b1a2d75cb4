"""Pins of the oracle's switch functions against the definitions of Section 2.2
and Section 4.2.

* Antisymmetry: S_K^{K'} = -S_{K'}^K on every interior face, and K is the
  q-side of the face exactly when S_K^{K'} = -1.
* Consistency (Section 4.2): |sum_i S_K^{K_i}| < |{K_i}|, i.e. every element has
  a face with S = +1 and one with S = -1.  The directional switch of R4 meets it
  on every element whose faces are all interior: the measure-weighted outward
  normals of a closed simplex sum to zero, so n . w takes both signs.
* The natural switch (S_K^{K'} = +1 when N(K) > N(K')) is inconsistent at the
  element with the largest enumeration, whose switches are all +1.
"""
import numpy as np
import pytest

from oracle.mesh import Topology
from synthetic import jittered_square, kuhn_cube


def _switches(t):
    S = [[] for _ in range(t.ne)]
    for f, (Ka, Kb, _, _) in enumerate(t.interior):
        S[Ka].append(int(t.S1[f]))
        S[Kb].append(-int(t.S1[f]))
    return S


@pytest.mark.parametrize("mesh", [jittered_square(10), kuhn_cube(3)], ids=["tri", "tet"])
def test_directional_switch_is_consistent_on_interior_elements(mesh):
    t = Topology(mesh)
    for f, (Ka, Kb, _, _) in enumerate(t.interior):
        assert t.qside[f] == (Ka if t.S1[f] == -1 else Kb)
        assert t.uside[f] == (Kb if t.S1[f] == -1 else Ka)
    S = _switches(t)
    full = [K for K in range(t.ne) if len(S[K]) == t.d + 1]
    assert len(full) > t.ne // 3
    for K in full:
        assert abs(sum(S[K])) < len(S[K]), K


def test_natural_switch_is_inconsistent_at_the_last_element():
    mesh = jittered_square(8)
    enum = np.random.default_rng(4).permutation(mesh.n_elements)
    t = Topology(mesh, switch_kind=1, enumeration=enum)
    S = _switches(t)
    top = int(np.argmax(enum))
    assert all(s == 1 for s in S[top]) and abs(sum(S[top])) == len(S[top])
    for f, (Ka, Kb, _, _) in enumerate(t.interior):
        assert t.S1[f] == (1 if enum[Ka] > enum[Kb] else -1)
