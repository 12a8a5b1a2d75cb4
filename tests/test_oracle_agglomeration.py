"""Pins of the oracle's agglomeration (Section 3.2, Algorithm 2; Section 3.1,
Algorithm 1): a hand-traced example (tests/golden/agglomeration_2x2.txt), the
SplitMix64 reference outputs behind the tie-break rule R9, partition and
connectivity (Section 3.1: every subset must be connected), determinism, and
the nested tree numbering."""
import os

import numpy as np
import pytest

from oracle.agglomerate import Hierarchy, greedy_agglomerate, splitmix64
from oracle.mesh import Topology
from synthetic import jittered_square, kuhn_cube

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _hier(mesh, levels, seed=0):
    t = Topology(mesh)
    return Hierarchy([list(map(int, e)) for e in mesh.elem], t.nbrs, levels, seed)


def test_splitmix64_reference_outputs():
    # first two outputs of the SplitMix64 generator started from state 0
    assert splitmix64(0) == 0xE220A8397B1DCDAF
    assert splitmix64(0x9E3779B97F4A7C15) == 0x6E789E6AA1B965F4


def test_hand_traced_example():
    expect = {}
    for line in open(os.path.join(GOLDEN, "agglomeration_2x2.txt")):
        if line.startswith("level"):
            tok = line.split()
            expect[int(tok[1])] = [int(x) for x in tok[3:]]
    H = _hier(jittered_square(2), 10)
    assert H.n_levels == 3
    for l, par in expect.items():
        assert H.parent[l] == par
    assert H.blocks[0] == [[2, 0, 3, 1], [5, 4, 7, 6]]


@pytest.mark.parametrize("mesh", [jittered_square(12), kuhn_cube(3)], ids=["tri", "tet"])
def test_partition_connected_and_deterministic(mesh):
    H = _hier(mesh, 10, seed=7)
    H2 = _hier(mesh, 10, seed=7)
    assert H.parent == H2.parent
    assert len(H.verts[-1]) == 1 or H.n_levels == 10
    for l in range(H.n_levels - 1):
        par = H.parent[l]
        n_c = len(H.verts[l + 1])
        assert sorted(set(par)) == list(range(n_c))          # every block non-empty
        for B, es in enumerate(H.blocks[l]):
            assert all(par[e] == B for e in es)
            # vertex-connected (R11): BFS over shared vertices inside the block
            seen, todo = {es[0]}, [es[0]]
            while todo:
                e = todo.pop()
                for e2 in es:
                    if e2 not in seen and set(H.verts[l][e]) & set(H.verts[l][e2]):
                        seen.add(e2); todo.append(e2)
            assert seen == set(es)
        # members of coarse elements partition the fine elements
        allm = sorted(m for mem in H.members[l + 1] for m in mem)
        assert allm == list(range(mesh.n_elements))


def test_tree_order_contiguous_children():
    H = _hier(jittered_square(10), 5)
    order = H.tree_order()
    for l in range(H.n_levels - 1):
        pos_c = {e: i for i, e in enumerate(order[l + 1])}
        parents_in_order = [pos_c[H.parent[l][e]] for e in order[l]]
        assert parents_in_order == sorted(parents_in_order)


def test_star_branch_groups_vertex_neighbourhood():
    # a single vertex star: the six triangles around the centre of a hexagon-like
    # patch all contain vertex 0 -> one block
    verts = [[0, 1, 2], [0, 2, 3], [0, 3, 4], [0, 4, 5], [0, 5, 6], [0, 6, 1]]
    nbrs = [[5, 1], [0, 2], [1, 3], [2, 4], [3, 5], [4, 0]]
    assert greedy_agglomerate(verts, nbrs, 0, 0) == [[0, 1, 2, 3, 4, 5]]
