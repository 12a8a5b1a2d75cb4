"""GPU parity of the p-multigrid front end (Section 4.4; reading R17: the CDG
operator rediscretised at degrees p, p-1, ..., 2 on the fine mesh, truncation
transfers between degrees, then the p = 1 agglomeration hierarchy) against the
oracle, called through the C ABI.  Tolerances as in test_gpu_parity: transfers
1e-13, V-cycle 1e-9 (dense coarsest solves on both sides agree to
cond(A_n) eps), full solves 1e-10 with iteration counts within one."""
import numpy as np
import pytest

from oracle.cdg import Level0
from oracle.gmres import gmres
from oracle.hierarchy import MGHierarchy
from oracle.solver import VCycle, pcg
from synthetic import jittered_square, kuhn_cube, sin_source
from tests.gpu_common import rel

pytestmark = pytest.mark.gpu

CASES = {
    "tri_p3_24": (lambda: jittered_square(24), dict(p=3, max_levels=5)),
    "tri_p2_16_neumann": (lambda: jittered_square(16, neumann_axes=(0,)), dict(p=2, max_levels=4)),
    "tet_p2_4": (lambda: kuhn_cube(4), dict(p=2, max_levels=4)),
}


def _t(x):
    import torch
    return torch.as_tensor(np.ascontiguousarray(x), device="cuda")


class Case:
    def __init__(self, mesh, kw):
        from paper_2012_08024_gb300 import Solver
        self.S = Solver(mesh, pmg=True, **kw).bind()
        self.L0 = Level0(mesh, kw["p"])
        self.H = MGHierarchy(self.L0, max_levels=kw["max_levels"], pmg=True)
        self.order = self.H.tree_order()

    def to_tree(self, l, x):
        npb = self.H.nps[l]
        return np.asarray(x).reshape(-1, npb)[self.order[l]].ravel()

    def to_work(self, l, x):
        npb = self.H.nps[l]
        y = np.empty((len(self.order[l]), npb))
        y[self.order[l]] = np.asarray(x).reshape(-1, npb)
        return y.ravel()


@pytest.fixture(scope="module", params=list(CASES))
def case(request):
    mk, kw = CASES[request.param]
    c = Case(mk(), kw)
    assert c.S.n_levels == c.H.n_levels and c.S.info["np_l"] == c.H.nps
    return c


def test_degree_transfers(case):
    import torch
    S, H = case.S, case.H
    rng = np.random.default_rng(0)
    for l in range(H.n_plevels):
        nf, nc = H.A[l].shape[0], H.A[l + 1].shape[0]
        r = rng.standard_normal(nf)
        bc = torch.empty(nc, dtype=torch.float64, device="cuda")
        S.restrict(l, _t(case.to_tree(l, r)), bc)
        assert rel(case.to_work(l + 1, bc.cpu().numpy()), H.L[l].T @ r) <= 1e-13
        xc = rng.standard_normal(nc)
        x0 = rng.standard_normal(nf)
        x = _t(case.to_tree(l, x0)).clone()
        S.prolong(l, _t(case.to_tree(l + 1, xc)), x)
        assert rel(case.to_work(l, x.cpu().numpy()), x0 + H.L[l] @ xc) <= 1e-13


def test_operators_and_smoother_per_level(case):
    import torch
    S, H = case.S, case.H
    rng = np.random.default_rng(1)
    for l in range(H.n_levels - 1):
        n = H.A[l].shape[0]
        x = rng.standard_normal(n)
        y = torch.empty(n, dtype=torch.float64, device="cuda")
        S.apply(l, _t(case.to_tree(l, x)), y)
        assert rel(case.to_work(l, y.cpu().numpy()), H.A[l] @ x) <= 1e-13


def test_vcycle(case):
    import torch
    S, H = case.S, case.H
    V = VCycle(H.A, H.L, H.nps, 1, 1)
    r = np.random.default_rng(3).standard_normal(H.A[0].shape[0])
    z = torch.empty(len(r), dtype=torch.float64, device="cuda")
    S.vcycle(_t(case.to_tree(0, r)), z)
    assert rel(case.to_work(0, z.cpu().numpy()), V.apply(r)) <= 1e-9


def test_full_solve(case):
    import scipy.sparse.linalg as spl
    S, H, L0 = case.S, case.H, case.L0
    xq, _, _ = S.quadrature_points()
    fq = sin_source(xq)
    u, hist, it, rc = S.solve(_t(fq))
    assert rc == 0 and hist[-1] <= 1e-10
    b = L0.rhs(fq)
    V = VCycle(H.A, H.L, H.nps, 1, 1)
    uo, ho, ito = pcg(H.A[0], b, V.apply, tol=1e-10)
    assert abs(it - ito) <= 1, (it, ito)
    ug = u.cpu().numpy().ravel()
    if it == ito:
        assert rel(ug, uo) <= 1e-10
    else:
        ud = spl.spsolve(H.A[0].tocsc(), b)
        assert rel(ug, ud) <= 1e-10
    assert np.linalg.norm(b - H.A[0] @ ug) <= 2e-10 * np.linalg.norm(b)


def test_pmg_cuts_iterations_and_works_with_gmres_and_fp32():
    from paper_2012_08024_gb300 import Solver
    mesh = jittered_square(32)
    kw = dict(p=3, max_levels=8, nu_pre=1, nu_post=1)
    its = {}
    for pmg in (False, True):
        S = Solver(mesh, pmg=pmg, **kw).bind()
        u, hist, it, rc = S.solve(_t(sin_source(S.quadrature_points()[0])))
        assert rc == 0
        its[pmg] = it
    assert its[True] < 0.85 * its[False], its
    # the paper's solver settings with the p-multigrid front end, FP64 and FP32 V-cycles
    L0 = Level0(mesh, 3)
    H = MGHierarchy(L0, max_levels=8, pmg=True)
    V = VCycle(H.A, H.L, H.nps, 0, 3)
    xq = L0.all_volume_points()
    b = L0.rhs(sin_source(xq))
    uo, ho, ito = gmres(H.A[0], b, V.apply, m=50, tol=1e-8)
    for prec in ("fp64", "fp32"):
        S = Solver(mesh, pmg=True, p=3, max_levels=8, nu_pre=0, nu_post=3, krylov="gmres", tol=1e-8,
                   precision=prec).bind()
        u, hist, it, rc = S.solve(_t(sin_source(S.quadrature_points()[0])))
        assert rc == 0 and abs(it - ito) <= (1 if prec == "fp64" else 3), (prec, it, ito)
        assert np.linalg.norm(b - H.A[0] @ u.cpu().numpy().ravel()) <= 2e-8 * np.linalg.norm(b)


def test_p1_pmg_is_the_plain_solver():
    from paper_2012_08024_gb300 import Solver
    mesh = jittered_square(12)
    Sa = Solver(mesh, p=1, max_levels=4, pmg=True).bind()
    Sb = Solver(mesh, p=1, max_levels=4).bind()
    assert Sa.info["n_plevels"] == 0
    fq = _t(sin_source(Sa.quadrature_points()[0]))
    ua, ha, ita, _ = Sa.solve(fq)
    ub, hb, itb, _ = Sb.solve(fq)
    assert ita == itb and np.array_equal(ua.cpu().numpy(), ub.cpu().numpy())
