"""The persistent V-cycle (persistent_vcycle): the whole cycle of Section 4.3
(Algorithm 3, reading R14) as one cooperative kernel with grid barriers
between its phases.  It runs the same arithmetic in the same order as the
per-phase kernels, so its V-cycle agrees with theirs to rounding (1e-14) and
its solves take the same iteration counts; batched solves of many meshes of
uneven size are checked against the oracle's PCG; every barrier wait is
bounded, and a host-set limit of 0 makes the solve return CDG_ETIMEOUT
without faulting the GPU, after which the handle solves normally again."""
import numpy as np
import pytest

from synthetic import batched_squares, jittered_square, kuhn_cube, sin_source
from tests.gpu_common import OracleCase, rel

pytestmark = pytest.mark.gpu


def _t(x):
    import torch
    return torch.tensor(np.ascontiguousarray(x), dtype=torch.float64, device="cuda")


@pytest.mark.parametrize("precision,nu", [("fp64", 1), ("fp64", 2), ("fp32", 2)])
def test_persistent_vcycle_equals_per_phase_kernels(precision, nu):
    import torch
    from paper_2012_08024_gb300 import Solver
    mesh = jittered_square(24)
    kw = dict(p=3, max_levels=4, nu_pre=nu, nu_post=nu, precision=precision)
    S1 = Solver(mesh, **kw).bind()
    S2 = Solver(mesh, persistent_vcycle=True, **kw).bind()
    n = S1.info["n_dofs"]
    r = torch.tensor(np.random.default_rng(9).standard_normal(n), device="cuda")
    z1, z2 = torch.empty_like(r), torch.empty_like(r)
    for _ in range(2):   # twice: the per-phase kernels keep their buffer roles across cycles
        S1.vcycle(r, z1)
        S2.vcycle(r, z2)
        torch.cuda.synchronize()
        assert rel(z2.cpu().numpy(), z1.cpu().numpy()) <= (1e-14 if precision == "fp64" else 1e-6)
    fq = _t(sin_source(S1.quadrature_points()[0]))
    u1, h1, it1, rc1 = S1.solve(fq)
    u2, h2, it2, rc2 = S2.solve(fq)
    assert rc1 == rc2 == 0 and abs(it1 - it2) <= (0 if precision == "fp64" else 1)
    assert rel(u2.cpu().numpy(), u1.cpu().numpy()) <= 1e-10
    assert S2.solve_graph()   # the cooperative launch sits inside the one-graph CG loop


def test_persistent_batched_matches_oracle():
    from oracle.solver import pcg
    from paper_2012_08024_gb300 import BatchSolver
    meshes = [jittered_square(n, seed=k) for k, n in enumerate((9, 14, 6, 11))]
    B = BatchSolver(meshes, p=2, max_levels=3, persistent_vcycle=True).bind()
    xq, _, _ = B.quadrature_points()
    fq = sin_source(xq)
    u, hists, its, rc = B.solve(_t(fq))
    assert rc == 0
    ub = u.cpu().numpy()
    for m, mesh in enumerate(meshes):
        oc = OracleCase(mesh, 2, 3)
        e0, e1 = B.elem_offsets[m], B.elem_offsets[m + 1]
        uo, ho, ito = pcg(oc.H.A[0], oc.L0.rhs(fq[e0:e1]), oc.V.apply, tol=1e-10)
        assert abs(int(its[m]) - ito) <= 1, (m, its[m], ito)
        assert rel(ub[e0:e1], uo.reshape(-1, ub.shape[1])) <= 1e-10


def test_persistent_batched_64_meshes_equals_per_phase():
    from paper_2012_08024_gb300 import BatchSolver
    meshes = batched_squares(64, 500, 20000, seed=1)
    out = []
    for pv in (False, True):
        B = BatchSolver(meshes, p=2, max_levels=4, persistent_vcycle=pv).bind()
        fq = _t(sin_source(B.quadrature_points()[0]))
        u, hists, its, rc = B.solve(fq)
        assert rc == 0
        out.append((u.cpu().numpy(), np.asarray(its)))
    assert np.abs(out[0][1] - out[1][1]).max() <= 1
    assert rel(out[1][0], out[0][0]) <= 1e-10


def test_persistent_falls_back_on_degree_steps():
    """A p-multigrid hierarchy changes n_p between levels: the per-phase
    kernels run instead, and the solve is unchanged."""
    from paper_2012_08024_gb300 import Solver
    mesh = jittered_square(12)
    kw = dict(p=3, max_levels=3, pmg=True)
    fq = _t(sin_source(Solver(mesh, **kw).quadrature_points()[0]))
    res = []
    for pv in (False, True):
        S = Solver(mesh, persistent_vcycle=pv, **kw).bind()
        res.append(S.solve(fq))
    assert res[0][3] == res[1][3] == 0 and res[0][2] == res[1][2]
    assert rel(res[1][0].cpu().numpy(), res[0][0].cpu().numpy()) <= 1e-14


def test_persistent_barrier_timeout_is_reported_and_recoverable():
    from paper_2012_08024_gb300 import CdgError, Solver
    mesh = kuhn_cube(4)
    S = Solver(mesh, p=2, max_levels=3, persistent_vcycle=True).bind()
    fq = _t(sin_source(S.quadrature_points()[0]))
    S.set_wait_limit(0)
    with pytest.raises(CdgError) as e:
        S.solve(fq)
    assert e.value.code == 6 and "grid barrier" in str(e.value)
    S.set_wait_limit(-1)
    u1, h1, it1, rc1 = S.solve(fq)
    S2 = Solver(mesh, p=2, max_levels=3).bind()
    u2, h2, it2, rc2 = S2.solve(fq)
    assert rc1 == rc2 == 0 and it1 == it2 and rel(u1.cpu().numpy(), u2.cpu().numpy()) <= 1e-10
