"""Differentiation of the solve on the GPU (cdg_solve_adjoint, cdg_rhs_adjoint,
cdg_kappa_gradient behind a torch.autograd.Function) against the oracle
adjoint (oracle/adjoint.py, direct solves) and central finite differences.

Tolerances: the gradient kernels evaluated on given (lambda, u) agree with the
oracle to 1e-12 (FP64 summation order); the full gradients of the
differentiable workload (smoothed log-normal kappa, target from another kappa)
agree with the oracle adjoint to 1e-9 with solves to 1e-12; finite differences
with h = 1e-6 on 20 random directions agree to 1e-5 of ||grad|| ||d||."""
import numpy as np
import pytest
import scipy.sparse.linalg as spl

from oracle.adjoint import kappa_gradient, rhs_gradient
from oracle.cdg import Level0
from synthetic import face_neighbors, kuhn_cube, sin_source, smoothed_lognormal_kappa
from tests.gpu_common import rel

pytestmark = pytest.mark.gpu


def _t(x):
    import torch
    return torch.tensor(np.ascontiguousarray(x), dtype=torch.float64, device="cuda")


def test_gradient_kernels_match_oracle():
    from paper_2012_08024_gb300 import Solver
    mesh = kuhn_cube(3)
    rng = np.random.default_rng(0)
    kappa = np.exp(0.5 * rng.standard_normal(mesh.n_elements))
    S = Solver(mesh, p=2, max_levels=3, kappa=kappa).bind()
    L0 = Level0(mesh, 2, kappa=kappa)
    n = mesh.n_elements * L0.np_
    lam, u = rng.standard_normal(n), rng.standard_normal(n)
    xq, xbq, _ = S.quadrature_points()
    gD = rng.standard_normal(xbq.shape[:2])
    g = S.kappa_gradient(_t(lam), _t(u), _t(gD)).cpu().numpy()
    assert rel(g, kappa_gradient(L0, lam, u, gD)) <= 1e-12
    g0 = S.kappa_gradient(_t(lam), _t(u)).cpu().numpy()
    assert rel(g0, kappa_gradient(L0, lam, u)) <= 1e-12
    gf = S.rhs_adjoint(_t(lam)).cpu().numpy()
    assert rel(gf, rhs_gradient(L0, lam)) <= 1e-13


def _workload(n):
    mesh = kuhn_cube(n)
    nb = face_neighbors(mesh)
    kappa = smoothed_lognormal_kappa(nb, seed=2)
    kstar = smoothed_lognormal_kappa(nb, seed=3)
    return mesh, kappa, kstar


def test_autograd_matches_oracle_adjoint():
    import torch
    from paper_2012_08024_gb300.autograd import CDGSolve, SolverCache
    mesh, kappa, kstar = _workload(4)
    opts = dict(p=2, max_levels=3, tol=1e-12, maxit=2000)
    cache = SolverCache(mesh, **opts)
    xq = cache.get(torch.tensor(kstar), "cuda").quadrature_points()[0]
    fq = _t(sin_source(xq))
    with torch.no_grad():
        ut = CDGSolve.apply(fq, torch.tensor(kstar, device="cuda"), cache)
    f = fq.clone().requires_grad_(True)
    k = torch.tensor(kappa, device="cuda", requires_grad=True)
    u = CDGSolve.apply(f, k, cache)
    L = ((u - ut) ** 2).sum()
    L.backward()
    # oracle: direct solves, own assembly, own adjoint
    L0s = Level0(mesh, 2, kappa=kstar)
    uts = spl.spsolve(L0s.matrix().tocsc(), L0s.rhs(sin_source(xq)))
    L0 = Level0(mesh, 2, kappa=kappa)
    A = L0.matrix().tocsc()
    uo = spl.spsolve(A, L0.rhs(sin_source(xq)))
    lam = spl.spsolve(A, 2 * (uo - uts))
    assert rel(u.detach().cpu().numpy(), uo) <= 1e-10
    assert rel(k.grad.cpu().numpy(), kappa_gradient(L0, lam, uo)) <= 1e-9
    assert rel(f.grad.cpu().numpy(), rhs_gradient(L0, lam)) <= 1e-9


def test_finite_differences_20_directions():
    import torch
    from paper_2012_08024_gb300.autograd import CDGSolve, SolverCache
    mesh, kappa, kstar = _workload(6)
    opts = dict(p=2, max_levels=4, tol=1e-12, maxit=2000, coarsen="primal")
    cache = SolverCache(mesh, **opts)
    xq = cache.get(torch.tensor(kstar), "cuda").quadrature_points()[0]
    fq = _t(sin_source(xq))
    with torch.no_grad():
        ut = CDGSolve.apply(fq, torch.tensor(kstar, device="cuda"), cache)

    def loss(kap):
        with torch.no_grad():
            u = CDGSolve.apply(fq, torch.tensor(kap, device="cuda"), cache)
            return float(((u - ut) ** 2).sum())
    k = torch.tensor(kappa, device="cuda", requires_grad=True)
    L = ((CDGSolve.apply(fq, k, cache) - ut) ** 2).sum()
    L.backward()
    g = k.grad.cpu().numpy()
    rng = np.random.default_rng(5)
    h = 1e-6
    for _ in range(20):
        d = rng.standard_normal(mesh.n_elements)
        fd = (loss(kappa + h * d) - loss(kappa - h * d)) / (2 * h)
        assert abs(fd - g @ d) <= 1e-5 * np.linalg.norm(g) * np.linalg.norm(d), (fd, g @ d)
