"""Pins of the oracle adjoint (oracle/adjoint.py):
* homogeneity: A_0 is linear in kappa with each term owned once, so
  sum_K kappa_K lambda^T dA_0/dkappa_K u = lambda^T A_0 u exactly;
* central finite differences of L = ||u - u_t||^2 with direct solves, in
  kappa (log-parametrised, kappa exp(h d)) and in f, with non-zero Dirichlet
  data (exercises db/dkappa), on a triangle and a tetrahedron mesh: with
  h = 1e-4 the truncation error is O(h^2) ~ 1e-8 and the solve noise ~1e-8, so
  the directional derivative must agree to 1e-6 of ||grad|| ||d||."""
import numpy as np
import pytest
import scipy.sparse.linalg as spl

from oracle.adjoint import kappa_gradient, rhs_gradient
from oracle.cdg import Level0
from synthetic import jittered_square, kuhn_cube


@pytest.mark.parametrize("dim", [2, 3])
def test_homogeneity(dim):
    mesh = jittered_square(5, neumann_axes=(0,)) if dim == 2 else kuhn_cube(2)
    rng = np.random.default_rng(0)
    kappa = np.exp(0.5 * rng.standard_normal(mesh.n_elements))
    L0 = Level0(mesh, 2 if dim == 2 else 1, kappa=kappa)
    A = L0.matrix()
    u, lam = rng.standard_normal(A.shape[0]), rng.standard_normal(A.shape[0])
    g = kappa_gradient(L0, lam, u)
    assert abs(-(kappa * g).sum() - lam @ (A @ u)) <= 1e-12 * abs(lam @ (A @ u))


def _loss_and_grads(mesh, p, kappa, fq, gD, ut):
    L0 = Level0(mesh, p, kappa=kappa)
    A = L0.matrix().tocsc()
    b = L0.rhs(fq, gD)
    u = spl.spsolve(A, b)
    r = u - ut
    lam = spl.spsolve(A, 2 * r)
    return L0, float(r @ r), kappa_gradient(L0, lam, u, gD), rhs_gradient(L0, lam)


@pytest.mark.parametrize("dim", [2, 3])
def test_finite_differences(dim):
    mesh = jittered_square(4, neumann_axes=(1,)) if dim == 2 else kuhn_cube(2)
    p = 2 if dim == 2 else 1
    rng = np.random.default_rng(1)
    kappa = np.exp(0.5 * rng.standard_normal(mesh.n_elements))
    L0 = Level0(mesh, p, kappa=kappa)
    fq = rng.standard_normal((mesh.n_elements, len(L0.vrule[1])))
    gD = rng.standard_normal((len(L0.topo.boundary), len(L0.frule[1])))
    # target from another coefficient field, as in the differentiable workload
    kstar = np.exp(0.5 * rng.standard_normal(mesh.n_elements))
    L0s = Level0(mesh, p, kappa=kstar)
    ut = spl.spsolve(L0s.matrix().tocsc(), L0s.rhs(fq, gD))
    _, L, gk, gf = _loss_and_grads(mesh, p, kappa, fq, gD, ut)
    h = 1e-4
    for k in range(4):
        d = rng.standard_normal(mesh.n_elements)
        Lp = _loss_and_grads(mesh, p, kappa * np.exp(h * d), fq, gD, ut)[1]
        Lm = _loss_and_grads(mesh, p, kappa * np.exp(-h * d), fq, gD, ut)[1]
        fd = (Lp - Lm) / (2 * h)
        an = gk @ (kappa * d)
        assert abs(fd - an) <= 1e-6 * np.linalg.norm(gk * kappa) * np.linalg.norm(d), (fd, an)
        df = rng.standard_normal(fq.shape)
        Lp = _loss_and_grads(mesh, p, kappa, fq + h * df, gD, ut)[1]
        Lm = _loss_and_grads(mesh, p, kappa, fq - h * df, gD, ut)[1]
        fd = (Lp - Lm) / (2 * h)
        an = (gf * df).sum()
        assert abs(fd - an) <= 1e-6 * np.linalg.norm(gf) * np.linalg.norm(df), (fd, an)
