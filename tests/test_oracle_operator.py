"""Pins of the oracle's level-0 CDG operator (Section 2) against what the
paper and the mathematics fix:

* symmetry and positive definiteness (Section 4: A is SPD for Poisson);
* smallest eigenvalue of the discrete Dirichlet Laplacian on the unit square
  (cube) close to 2 pi^2 (3 pi^2), the continuous value;
* polynomial reproduction: with f = -Lap P, g_D = P, g_N = dP/dn the discrete
  solution is P for every P of degree <= p (CDG is consistent), which pins the
  signs of all consistency, source and boundary terms (reading R1);
* energy of piecewise constants in closed form: for p = 1 the lifting of a
  unit jump on face f of the q-side triangle K has energy 3|f|^2/|K| (2D) and
  8|f|^2/(3|K|) (3D), from the P1 mass matrix |K|/((d+1)(d+2)) (I + 11^T), so
  a(u,u) = sum_f kappa_q c_d |f|^2/|K_q| [[u]]^2 + C_D sum_{Gamma_D} kappa |f| u^2;
  this pins the lifting term, the q-side choice (eq. edge_flux_interior), C_D
  and h_avg (R6);
* L2 convergence of order p+1 for u = prod sin(pi x_i);
* compactness of A (eq. primal_form) and the second-neighbour pattern of C
  (Section 4.2): the (K_i, K_n) block of C is non-zero exactly when the element
  K_j between them has S_{K_i}^{K_j} = 1 and S_{K_j}^{K_n} = -1.
"""
import math

import numpy as np
import pytest
import scipy.sparse.linalg as spl

from oracle.cdg import Level0
from oracle.hierarchy import MGHierarchy
from oracle.quadrature import simplex_rule, map_simplex
from synthetic import jittered_square, kuhn_cube, sin_source, sin_solution


def test_symmetric_positive_definite():
    for mesh, p in ((jittered_square(4, neumann_axes=(0,)), 2), (kuhn_cube(1), 1)):
        A = Level0(mesh, p).matrix().toarray()
        assert np.abs(A - A.T).max() <= 1e-14 * np.abs(A).max()
        assert np.linalg.eigvalsh(A).min() > 0


def test_smallest_eigenvalue_is_laplace_eigenvalue():
    A = Level0(jittered_square(8), 2).matrix().toarray()
    lam = np.linalg.eigvalsh(A).min()
    assert abs(lam / (2 * math.pi ** 2) - 1) < 1e-3
    A3 = Level0(kuhn_cube(3), 2).matrix().toarray()
    lam3 = np.linalg.eigvalsh(A3).min()
    assert abs(lam3 / (3 * math.pi ** 2) - 1) < 2e-2


def _poly2(x):
    X, Y = x[..., 0], x[..., 1]
    return 0.3 + X - 0.7 * Y + 0.5 * X * Y + 0.25 * X ** 2 - 0.4 * Y ** 2


def _poly2_grad(x):
    X, Y = x[..., 0], x[..., 1]
    return np.stack([1 + 0.5 * Y + 0.5 * X, -0.7 + 0.5 * X - 0.8 * Y], axis=-1)


def _project(L0, fun):
    out = np.zeros((L0.topo.ne, L0.np_))
    for K in range(L0.topo.ne):
        x, w = L0.volume_points(K)
        out[K] = (L0.bases[K].eval(x) * (w * fun(x))[:, None]).sum(0)
    return out.ravel()


@pytest.mark.parametrize("p,neumann", [(2, ()), (2, (0,)), (3, (1,)), (1, (1,))])
def test_polynomial_reproduction_2d(p, neumann):
    if p == 1:
        P = lambda x: 0.3 + x[..., 0] - 0.7 * x[..., 1]
        dP = lambda x: np.broadcast_to(np.array([1.0, -0.7]), x.shape)
        lapP = 0.0
    else:
        P, dP, lapP = _poly2, _poly2_grad, 0.5 - 0.8
    mesh = jittered_square(5, neumann_axes=neumann)
    L0 = Level0(mesh, p, gamma=1e4)
    fq = np.full((L0.topo.ne, len(L0.vrule[1])), -lapP)
    xb = L0.all_boundary_points()
    gD = P(xb)
    nrm = np.array(L0.topo.bf_n)[:, None, :]
    gN = (dP(xb) * nrm).sum(-1)
    b = L0.rhs(fq, gD, gN)
    u = spl.spsolve(L0.matrix().tocsc(), b)
    ref = _project(L0, P)
    assert np.linalg.norm(u - ref) <= 1e-10 * np.linalg.norm(ref)


def test_polynomial_reproduction_3d():
    P = lambda x: 0.2 + x[..., 0] - 0.5 * x[..., 1] + 0.8 * x[..., 2]
    mesh = kuhn_cube(2, neumann_axes=(2,))
    L0 = Level0(mesh, 1)
    fq = np.zeros((L0.topo.ne, len(L0.vrule[1])))
    xb = L0.all_boundary_points()
    nrm = np.array(L0.topo.bf_n)[:, None, :]
    gN = (np.array([1.0, -0.5, 0.8]) * nrm).sum(-1) * np.ones(xb.shape[:2])
    b = L0.rhs(fq, P(xb), gN)
    u = spl.spsolve(L0.matrix().tocsc(), b)
    ref = _project(L0, P)
    assert np.linalg.norm(u - ref) <= 1e-10 * np.linalg.norm(ref)


@pytest.mark.parametrize("dim", [2, 3])
def test_piecewise_constant_energy_closed_form(dim):
    mesh = jittered_square(4, neumann_axes=(0,)) if dim == 2 else kuhn_cube(2)
    rng = np.random.default_rng(3)
    kappa = np.exp(rng.standard_normal(mesh.n_elements))
    L0 = Level0(mesh, 1, gamma=50.0, kappa=kappa)
    A = L0.matrix()
    t = L0.topo
    c = rng.standard_normal(t.ne)
    u = np.zeros((t.ne, L0.np_))
    u[:, 0] = c * np.sqrt(t.vol)          # phi_0 = 1/sqrt(|K|)
    u = u.ravel()
    cd = 3.0 if dim == 2 else 8.0 / 3.0
    expect = 0.0
    for f, (Ka, Kb, _, _) in enumerate(t.interior):
        q = t.qside[f]
        expect += kappa[q] * cd * t.if_meas[f] ** 2 / t.vol[q] * (c[Ka] - c[Kb]) ** 2
    for bf, (K, l, tag) in enumerate(t.boundary):
        if tag == 0:
            expect += kappa[K] * L0.C_D * t.bf_meas[bf] * c[K] ** 2
    assert abs(u @ (A @ u) - expect) <= 1e-12 * expect


def _l2_error(L0, u):
    rp, rw = simplex_rule(L0.d, 2 * L0.p + 6)
    err = 0.0
    U = u.reshape(L0.topo.ne, L0.np_)
    for K in range(L0.topo.ne):
        x, w = map_simplex(L0.topo.simplex(K), rp, rw)
        err += np.sum(w * (L0.bases[K].eval(x) @ U[K] - sin_solution(x)) ** 2)
    return math.sqrt(err)


@pytest.mark.parametrize("dim,p,ns", [(2, 1, (4, 8, 16)), (2, 2, (4, 8, 16)), (3, 1, (2, 4, 8))])
def test_l2_convergence_order(dim, p, ns):
    errs = []
    for n in ns:
        mesh = jittered_square(n) if dim == 2 else kuhn_cube(n)
        L0 = Level0(mesh, p)
        b = L0.rhs(sin_source(L0.all_volume_points()))
        u = spl.spsolve(L0.matrix().tocsc(), b)
        errs.append(_l2_error(L0, u))
    rate = math.log2(errs[-2] / errs[-1])
    assert abs(rate - (p + 1)) < 0.25, (errs, rate)


def test_compact_A_and_second_neighbour_pattern_of_C():
    mesh = jittered_square(6)
    L0 = Level0(mesh, 1)
    H = MGHierarchy(L0, max_levels=1)
    t, npb = L0.topo, L0.np_
    A, C = H.A[0].tocsr(), H.C[0].tocsr()
    nb = [set(x) for x in t.nbrs]
    qfaces = {}          # element -> set of neighbours across faces where it is the q-side
    for f in range(len(t.interior)):
        qfaces.setdefault(int(t.qside[f]), set()).add(int(t.uside[f]))

    def blocknorm(M, i, j):
        return np.abs(M[i * npb:(i + 1) * npb, j * npb:(j + 1) * npb].toarray()).max()
    scale = np.abs(C).max()
    for i in range(t.ne):
        for n_ in range(t.ne):
            if n_ == i or n_ in nb[i]:
                continue
            assert blocknorm(A, i, n_) == 0.0
            # K_j with S_{K_i}^{K_j} = 1 (K_j is the q-side of (i, j)) and
            # S_{K_j}^{K_n} = -1 (K_j is the q-side of (j, n))
            predicted = any(i in qfaces.get(j, ()) and n_ in qfaces.get(j, ()) for j in nb[i] & nb[n_])
            assert (blocknorm(C, i, n_) > 1e-12 * scale) == predicted, (i, n_)
