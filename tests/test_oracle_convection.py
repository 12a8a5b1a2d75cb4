"""Pins of the oracle's convection-diffusion operator (Section 5,
convection-diffusion; R18: -div(kappa grad u) + beta v . grad u = f with the
convection in upwind DG form and constant v).

* Consistency: for a polynomial P of degree <= p with f = -lap P + beta v.grad P,
  g_D = P and g_N = dP/dn the discrete solution is P itself (upwind DG and
  CDG are both consistent), on meshes with Dirichlet and Neumann sides.
* Upwind dissipation: for constant v, u^T (B + B^T) u equals the sum over
  interior faces of |beta v.n| int [[u]]^2, plus |beta v.n| int u^2 over
  Dirichlet faces and beta v.n int u^2 over Neumann faces (B the convection
  part; integrate u v.grad u by parts).
* beta = 0 is the Poisson operator.
"""
import numpy as np
import pytest
import scipy.sparse.linalg as spl

from oracle.cdg import Level0, blocks_to_csr
from synthetic import jittered_square, kuhn_cube


def _project(L0, fun):
    out = np.zeros((L0.topo.ne, L0.np_))
    for K in range(L0.topo.ne):
        x, w = L0.volume_points(K)
        out[K] = (L0.bases[K].eval(x) * (w * fun(x))[:, None]).sum(0)
    return out.ravel()


def _poly(x):
    X, Y = x[..., 0], x[..., 1]
    return 0.4 + X - 0.6 * Y + 0.5 * X * X - 0.3 * X * Y + 0.8 * Y * Y


def _poly_grad(x):
    X, Y = x[..., 0], x[..., 1]
    return np.stack([1.0 + X - 0.3 * Y, -0.6 - 0.3 * X + 1.6 * Y], axis=-1)


@pytest.mark.parametrize("beta,vel,neumann", [(1.0, (1.0, 0.0), ()), (10.0, (1.0, 0.3), (0,)),
                                               (100.0, (0.6, -0.8), (1,))])
def test_polynomial_reproduction(beta, vel, neumann):
    mesh = jittered_square(5, neumann_axes=neumann)
    L0 = Level0(mesh, 2, beta=beta, velocity=vel)
    xv = L0.all_volume_points()
    lap = 1.0 + 1.6
    fq = -lap + beta * (_poly_grad(xv) @ np.asarray(vel))
    xb = L0.all_boundary_points()
    nrm = np.array(L0.topo.bf_n)[:, None, :]
    gN = (_poly_grad(xb) * nrm).sum(-1)
    b = L0.rhs(fq, _poly(xb), gN)
    u = spl.spsolve(L0.matrix().tocsc(), b)
    ref = _project(L0, _poly)
    assert np.linalg.norm(u - ref) <= 1e-10 * np.linalg.norm(ref)


def test_polynomial_reproduction_3d():
    P = lambda x: 0.2 + x[..., 0] - 0.5 * x[..., 1] + 0.8 * x[..., 2]
    g = np.array([1.0, -0.5, 0.8])
    vel = np.array([0.3, 1.0, -0.2])
    mesh = kuhn_cube(2, neumann_axes=(2,))
    L0 = Level0(mesh, 1, beta=5.0, velocity=vel)
    fq = np.full((L0.topo.ne, len(L0.vrule[1])), 5.0 * float(g @ vel))
    xb = L0.all_boundary_points()
    nrm = np.array(L0.topo.bf_n)[:, None, :]
    gN = (g * nrm).sum(-1) * np.ones(xb.shape[:2])
    u = spl.spsolve(L0.matrix().tocsc(), L0.rhs(fq, P(xb), gN))
    ref = _project(L0, P)
    assert np.linalg.norm(u - ref) <= 1e-10 * np.linalg.norm(ref)


@pytest.mark.parametrize("neumann", [(), (0,)])
def test_upwind_dissipation_identity(neumann):
    mesh = jittered_square(4, neumann_axes=neumann)
    beta, vel = 7.0, np.array([0.8, 0.6])
    L0 = Level0(mesh, 2, beta=beta, velocity=vel)
    t = L0.topo
    B = blocks_to_csr(L0.convection_blocks(), t.ne, t.ne, L0.np_, L0.np_).toarray()
    u = np.random.default_rng(2).standard_normal(t.ne * L0.np_)
    U = u.reshape(t.ne, L0.np_)
    expect = 0.0
    for f, (K1, K2, _, _) in enumerate(t.interior):
        x, w = L0.interior_face_points(f)
        jump = L0.bases[K1].eval(x) @ U[K1] - L0.bases[K2].eval(x) @ U[K2]
        expect += abs(beta * float(vel @ t.if_n[f])) * (w * jump ** 2).sum()
    for bf, (K, l, tag) in enumerate(t.boundary):
        vn = beta * float(vel @ t.bf_n[bf])
        x, w = L0.boundary_face_points(bf)
        # Dirichlet faces: |v.n| (inflow data moved to the right-hand side);
        # Neumann faces keep the trace u_K, so inflow counts negatively
        expect += (abs(vn) if tag == 0 else vn) * (w * (L0.bases[K].eval(x) @ U[K]) ** 2).sum()
    assert abs(u @ (B + B.T) @ u - expect) <= 1e-11 * abs(expect)


def test_beta_zero_is_poisson():
    mesh = jittered_square(4)
    A0 = Level0(mesh, 2).matrix()
    A1 = Level0(mesh, 2, beta=0.0, velocity=(1.0, 0.0)).matrix()
    assert abs(A0 - A1).max() == 0.0
