"""Batched handles (host side, CPU): the batch's level operators, transfers and
tree order are the block-diagonal union of the meshes' own set-ups, bit for
bit, and the offsets / quadrature points concatenate the meshes in order."""
import numpy as np
import pytest

from synthetic import jittered_square


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2012_08024_gb300 import build
    build.build()


def test_batch_is_block_diagonal_union():
    from paper_2012_08024_gb300 import BatchSolver, Solver
    meshes = [jittered_square(n, seed=k) for k, n in enumerate((6, 9, 4))]
    B = BatchSolver(meshes, p=2, max_levels=3)
    singles = [Solver(m, p=2, max_levels=3) for m in meshes]
    assert B.n_meshes == 3
    assert list(B.elem_offsets) == list(np.cumsum([0] + [m.n_elements for m in meshes]))
    for l in range(B.n_levels):
        eb = B.export_level(l)
        ro = 0
        bo = 0
        for S, m in zip(singles, meshes):
            es = S.export_level(l)
            n = len(es["perm"])
            rows = slice(ro, ro + n)
            assert np.array_equal(eb["rowptr"][ro:ro + n + 1] - eb["rowptr"][ro], es["rowptr"])
            nb = es["rowptr"][-1]
            assert np.array_equal(eb["col"][bo:bo + nb], es["col"] + ro)
            assert np.array_equal(eb["val"][bo:bo + nb], es["val"])
            if l + 1 < B.n_levels:
                assert np.array_equal(eb["L"][rows], es["L"])
            if l == 0:
                eo = B.elem_offsets[singles.index(S)]
                assert np.array_equal(eb["perm"][rows], es["perm"] + eo)
            ro += n
            bo += nb
    xq, xbq, _ = B.quadrature_points()
    xs = np.concatenate([S.quadrature_points()[0] for S in singles])
    assert np.array_equal(xq, xs)


def test_batch_rejects_mismatched_levels():
    from paper_2012_08024_gb300 import BatchSolver, CdgError
    with pytest.raises(CdgError):
        BatchSolver([jittered_square(8), jittered_square(1)], p=1, max_levels=4)
