"""Batched solves (many meshes per handle, one launch per kernel for all of
them): each mesh's result equals its own single-mesh solve (iterations within
one, relative L2 1e-10: the per-mesh dot products are summed in a different
chunking) and, for small meshes, the oracle's PCG solution (1e-10)."""
import numpy as np
import pytest

from synthetic import batched_squares, jittered_square, sin_source
from tests.gpu_common import OracleCase, rel

pytestmark = pytest.mark.gpu


def _t(x):
    import torch
    return torch.tensor(np.ascontiguousarray(x), dtype=torch.float64, device="cuda")


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_batch_matches_single_solves(precision):
    from paper_2012_08024_gb300 import BatchSolver, Solver
    meshes = [jittered_square(n, seed=k) for k, n in enumerate((16, 23, 12, 30, 19))]
    kw = dict(p=2, max_levels=4, precision=precision)
    B = BatchSolver(meshes, **kw).bind()
    xq, _, _ = B.quadrature_points()
    u, hists, its, rc = B.solve(_t(sin_source(xq)))
    assert rc == 0
    ub = u.cpu().numpy()
    for m, mesh in enumerate(meshes):
        S = Solver(mesh, **kw).bind()
        xs, _, _ = S.quadrature_points()
        us, hs, it, rcs = S.solve(_t(sin_source(xs)))
        e0, e1 = B.elem_offsets[m], B.elem_offsets[m + 1]
        assert abs(int(its[m]) - it) <= 1 and hists[m][-1] <= 1e-10
        assert rel(ub[e0:e1], us.cpu().numpy()) <= 1e-10


def test_batch_matches_oracle():
    from oracle.solver import pcg
    from paper_2012_08024_gb300 import BatchSolver
    meshes = [jittered_square(6, seed=1), jittered_square(9, seed=2)]
    B = BatchSolver(meshes, p=2, max_levels=3).bind()
    xq, _, _ = B.quadrature_points()
    fq = sin_source(xq)
    u, hists, its, rc = B.solve(_t(fq))
    ub = u.cpu().numpy()
    for m, mesh in enumerate(meshes):
        oc = OracleCase(mesh, 2, 3)
        e0, e1 = B.elem_offsets[m], B.elem_offsets[m + 1]
        b = oc.L0.rhs(fq[e0:e1])
        uo, ho, ito = pcg(oc.H.A[0], b, oc.V.apply, tol=1e-10)
        assert abs(int(its[m]) - ito) <= 1
        if int(its[m]) != ito:
            uo, _, _ = pcg(oc.H.A[0], b, oc.V.apply, tol=0.0, maxit=int(its[m]))
        assert rel(ub[e0:e1], uo) <= 1e-10


def test_64_mesh_workload_converges():
    from paper_2012_08024_gb300 import BatchSolver
    meshes = batched_squares(64, 500, 20000, seed=1)
    B = BatchSolver(meshes, p=2, max_levels=4).bind()
    xq, _, _ = B.quadrature_points()
    u, hists, its, rc = B.solve(_t(sin_source(xq)))
    assert rc == 0 and B.n_meshes == 64
    assert all(h[-1] <= 1e-10 for h in hists)
