"""GPU parity of the convection-diffusion solve (Section 5; R18: upwind DG
convection, non-symmetric A_0) with GMRES(m) right-preconditioned by the
V-cycle, against the oracle.  Tolerances as in test_gpu_gmres."""
import numpy as np
import pytest

from oracle.cdg import Level0
from oracle.gmres import gmres
from oracle.hierarchy import MGHierarchy
from oracle.solver import VCycle
from synthetic import jittered_square, kuhn_cube
from tests.gpu_common import rel

pytestmark = pytest.mark.gpu


def _t(x):
    import torch
    return torch.as_tensor(np.ascontiguousarray(x), device="cuda")


CASES = {
    "tri_p1_beta1": (lambda: jittered_square(20), dict(p=1, beta=1.0, velocity=(1.0, 0.0))),
    "tri_p1_beta100": (lambda: jittered_square(20), dict(p=1, beta=100.0, velocity=(1.0, 0.0))),
    "tri_p2_beta10_neumann": (lambda: jittered_square(12, neumann_axes=(1,)),
                              dict(p=2, beta=10.0, velocity=(0.8, 0.6))),
    "tet_p1_beta5": (lambda: kuhn_cube(4), dict(p=1, beta=5.0, velocity=(0.3, 1.0, -0.2))),
}


@pytest.fixture(scope="module", params=list(CASES))
def case(request):
    from paper_2012_08024_gb300 import Solver
    mk, kw = CASES[request.param]
    mesh = mk()
    S = Solver(mesh, nu_pre=0, nu_post=3, max_levels=16, krylov="gmres", tol=1e-8, maxit=500, **kw).bind()
    L0 = Level0(mesh, kw["p"], beta=kw["beta"], velocity=kw["velocity"])
    H = MGHierarchy(L0, max_levels=16)
    assert S.n_levels == H.n_levels
    return S, L0, H


def test_rhs_with_inflow_data(case):
    S, L0, H = case
    xq, xbq, _ = S.quadrature_points()
    rng = np.random.default_rng(4)
    fq, gD, gN = (rng.standard_normal(xq.shape[:2]), rng.standard_normal(xbq.shape[:2]),
                  rng.standard_normal(xbq.shape[:2]))
    b = S.rhs(_t(fq), _t(gD), _t(gN))
    assert rel(b.cpu().numpy(), L0.rhs(fq, gD, gN)) <= 1e-13


def test_gmres_matches_oracle(case):
    S, L0, H = case
    xq, _, _ = S.quadrature_points()
    fq = np.ones(xq.shape[:2])                  # f = 1, zero Dirichlet data (Section 5)
    u, hist, it, rc = S.solve(_t(fq))
    assert rc == 0
    b = L0.rhs(fq)
    V = VCycle(H.A, H.L, L0.np_, 0, 3)
    uo, ho, ito = gmres(H.A[0], b, V.apply, m=50, tol=1e-8, maxit=500)
    assert abs(it - ito) <= 1, (it, ito)
    k = min(it, ito)
    ho = np.asarray(ho)
    assert np.all(np.abs(hist[:k] - ho[:k]) <= 1e-6 * ho[:k] + 1e-13)
    ug = u.cpu().numpy().ravel()
    assert np.linalg.norm(b - H.A[0] @ ug) <= 2e-8 * np.linalg.norm(b)
    if it == ito:
        assert rel(ug, uo) <= 1e-9


def test_polynomial_reproduction_on_the_device():
    from paper_2012_08024_gb300 import Solver
    mesh = jittered_square(10, neumann_axes=(0,))
    beta, vel = 20.0, np.array([1.0, 0.4])
    S = Solver(mesh, p=2, nu_pre=0, nu_post=3, max_levels=16, krylov="gmres", tol=1e-13, maxit=400,
               beta=beta, velocity=tuple(vel)).bind()
    L0 = Level0(mesh, 2, beta=beta, velocity=vel)
    P = lambda x: 0.4 + x[..., 0] - 0.6 * x[..., 1] + 0.5 * x[..., 0] ** 2 - 0.3 * x[..., 0] * x[..., 1]
    dP = lambda x: np.stack([1.0 + x[..., 0] - 0.3 * x[..., 1], -0.6 - 0.3 * x[..., 0]], axis=-1)
    xq, xbq, _ = S.quadrature_points()
    fq = -1.0 + beta * (dP(xq) @ vel)
    nrm = np.array(L0.topo.bf_n)[:, None, :]
    u, hist, it, rc = S.solve(_t(fq), _t(P(xbq)), _t((dP(xbq) * nrm).sum(-1)))
    assert rc == 0
    ref = np.zeros((L0.topo.ne, L0.np_))
    for K in range(L0.topo.ne):
        x, w = L0.volume_points(K)
        ref[K] = (L0.bases[K].eval(x) * (w * P(x))[:, None]).sum(0)
    assert rel(u.cpu().numpy(), ref) <= 1e-9


def test_fp32_vcycle_and_no_adjoint():
    from paper_2012_08024_gb300 import CdgError, Solver
    mesh = jittered_square(24)
    kw = dict(p=1, nu_pre=0, nu_post=3, max_levels=16, krylov="gmres", tol=1e-10, beta=10.0, velocity=(1.0, 0.0))
    S64 = Solver(mesh, **kw).bind()
    S32 = Solver(mesh, precision="fp32", **kw).bind()
    fq = _t(np.ones(S64.quadrature_points()[0].shape[:2]))
    u64, h64, it64, rc64 = S64.solve(fq)
    u32, h32, it32, rc32 = S32.solve(fq)
    assert rc64 == rc32 == 0 and abs(it32 - it64) <= 2
    assert rel(u32.cpu().numpy(), u64.cpu().numpy()) <= 1e-8
    with pytest.raises(CdgError):
        S64.solve_adjoint(u64)


def test_small_beta_leaves_the_iterations_unchanged():
    """Section 5: the preconditioner is nearly unaffected by small beta."""
    from paper_2012_08024_gb300 import Solver
    mesh = jittered_square(64)
    its = {}
    for beta in (0.0, 1.0):
        S = Solver(mesh, p=1, nu_pre=0, nu_post=3, max_levels=16, krylov="gmres", tol=1e-8, maxit=2000,
                   beta=beta, velocity=(1.0, 0.0)).bind()
        u, hist, it, rc = S.solve(_t(np.ones(S.quadrature_points()[0].shape[:2])))
        assert rc == 0
        its[beta] = it
    assert abs(its[1.0] - its[0.0]) <= 3, its
