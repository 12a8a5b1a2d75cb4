"""Parity at the full benchmark sizes, in the launch configurations bench.py
times, through properties that hold at any size and outputs the oracle can
compute element by element.

* Polynomial reproduction (consistency of the CDG discretisation, Section 2):
  with f = -lap P and g_D = P for a polynomial P of degree <= p the discrete
  solution is the L2 projection of P on every element.  The projection of a
  sampled element is computed independently with the oracle's basis and
  quadrature for that element alone.  Checked for the 512 x 512 p = 3 FP64
  solve (7 levels, V(2,2)) and the 48^3 x 6 p = 2 solve with the FP32 V-cycle
  (flux coarsening behind the p-multigrid front end, V(2,2)).
* The 256-column solve on the 158 x 158 x 2 mesh (BF16 blocks, tensor-core
  sweeps) against single-column FP64 solves of sampled columns, and the
  64-mesh batch against single-mesh solves of sampled meshes.
* The 24^3 x 6 differentiable workload: adjoint gradient against central finite
  differences in 20 directions.
"""
import numpy as np
import pytest

from oracle.basis import Basis
from oracle.quadrature import map_simplex, simplex_rule
from synthetic import batched_squares, jittered_square, kuhn_cube, sin_source, sine_combination_sources
from tests.gpu_common import rel

pytestmark = pytest.mark.gpu


def _t(x):
    import torch
    return torch.as_tensor(np.ascontiguousarray(x), device="cuda")


def _poly2d(x):
    X, Y = x[..., 0], x[..., 1]
    return (0.3 + X - 0.7 * Y + 0.5 * X * X - 0.4 * X * Y + 0.2 * Y * Y + 0.3 * X ** 3 - 0.2 * X * X * Y
            + 0.1 * X * Y * Y - 0.25 * Y ** 3)


def _lap_poly2d(x):      # P_xx + P_yy
    X, Y = x[..., 0], x[..., 1]
    return (1.0 + 1.8 * X - 0.4 * Y) + (0.4 + 0.2 * X - 1.5 * Y)


def _poly3d(x):
    X, Y, Z = x[..., 0], x[..., 1], x[..., 2]
    return 0.2 + X - 0.5 * Y + 0.8 * Z + 0.3 * X * X - 0.2 * Y * Z + 0.4 * Z * Z


def _projection(mesh, K, p, fun):
    """c_i = int_K fun phi_i, phi the orthonormal basis of element K (oracle)."""
    s = mesh.xyz[mesh.elem[K]]
    B = Basis([s], p)
    x, w = map_simplex(s, *simplex_rule(mesh.dim, 2 * p + 2))
    return (B.eval(x) * (w * fun(x))[:, None]).sum(0)


def _reproduction(mesh, S, p, fun, lap, nsample=200):
    xq, xbq, _ = S.quadrature_points()
    u, hist, it, rc = S.solve(_t(-lap(xq)), _t(fun(xbq)))
    assert rc == 0 and hist[-1] <= 1e-12, (rc, hist[-3:])
    U = u.cpu().numpy()
    rng = np.random.default_rng(11)
    ks = rng.choice(mesh.n_elements, size=nsample, replace=False)
    ref = np.stack([_projection(mesh, int(K), p, fun) for K in ks])
    return rel(U[ks], ref), it


def test_512_square_p3_fp64_reproduces_cubics():
    from paper_2012_08024_gb300 import Solver
    mesh = jittered_square(512)
    S = Solver(mesh, p=3, max_levels=7, nu_pre=2, nu_post=2, tol=1e-12, maxit=500).bind()
    err, it = _reproduction(mesh, S, 3, _poly2d, _lap_poly2d)
    print(f"512^2 p=3 FP64: {it} iterations, sampled projection error {err:.2e}")
    assert err <= 1e-8, err


def test_48_cube_p2_fp32_vcycle_reproduces_quadratics():
    """The 48^3 x 6 workload as bench.py runs it: flux coarsening (Section 4.1)
    behind the p-multigrid front end (Section 4.4), V(2,2), FP32 V-cycle."""
    from paper_2012_08024_gb300 import Solver
    mesh = kuhn_cube(48)
    S = Solver(mesh, p=2, max_levels=6, nu_pre=2, nu_post=2, coarsen="flux", pmg=True, precision="fp32",
               tol=1e-12, maxit=500).bind()
    err, it = _reproduction(mesh, S, 2, _poly3d, lambda x: np.full(x.shape[:-1], 1.4))
    print(f"48^3 p=2 FP32 V-cycle: {it} iterations, sampled projection error {err:.2e}")
    assert err <= 1e-8, err


def test_256_columns_against_single_solves():
    import torch
    from paper_2012_08024_gb300 import Solver
    mesh = jittered_square(158)
    R = 256
    kw = dict(p=3, max_levels=5, nu_pre=2, nu_post=2)
    SM = Solver(mesh, precision="bf16", nrhs=R, **kw).bind()
    S1 = Solver(mesh, **kw).bind()
    xq, _, _ = SM.quadrature_points()
    fq = sine_combination_sources(xq, R, mmax=8, seed0=0)
    U, hists, its, rc = SM.solve_multi(torch.tensor(fq, device="cuda"))
    assert rc == 0 and all(h[-1] <= 1e-10 for h in hists)
    for r in (0, 127, 128, 255):          # both 128-column tensor-core tiles, first and last columns
        u1, h1, it1, rc1 = S1.solve(_t(fq[r]))
        assert rc1 == 0
        assert rel(U[r].cpu().numpy(), u1.cpu().numpy()) <= 2e-9, r


def test_64_mesh_batch_against_single_meshes():
    from paper_2012_08024_gb300 import BatchSolver, Solver
    meshes = batched_squares(64, 500, 20000, seed=1)
    B = BatchSolver(meshes, p=2, max_levels=4).bind()
    xq, _, _ = B.quadrature_points()
    fq = sin_source(xq)
    u, hists, its, rc = B.solve(_t(fq))
    assert rc == 0
    eo = B.elem_offsets
    ub = u.cpu().numpy()
    for m in (0, 17, 40, 63):
        S = Solver(meshes[m], p=2, max_levels=4).bind()
        us, hs, its1, rc1 = S.solve(_t(fq[eo[m]:eo[m + 1]]))
        assert rc1 == 0 and abs(its1 - its[m]) <= 1
        assert rel(ub[eo[m]:eo[m + 1]], us.cpu().numpy()) <= 1e-9, m


def test_24_cube_gradient_20_fd_directions():
    """The differentiable 24^3 x 6 workload as bench.py runs it (p = 2, 5 levels,
    primal coarsening): dL/dkappa from the adjoint against central finite
    differences (h = 1e-6) in 20 random directions, each one two fresh set-ups of
    the whole hierarchy (about 2.5 s each)."""
    import torch
    from paper_2012_08024_gb300.autograd import CDGSolve, SolverCache
    from synthetic import face_neighbors, smoothed_lognormal_kappa
    mesh = kuhn_cube(24)
    nb = face_neighbors(mesh)
    kappa = smoothed_lognormal_kappa(nb, seed=2)
    kstar = smoothed_lognormal_kappa(nb, seed=3)
    cache = SolverCache(mesh, p=2, max_levels=5, coarsen="primal", tol=1e-12, maxit=2000)
    xq = cache.get(torch.tensor(kstar), "cuda").quadrature_points()[0]
    fq = _t(sin_source(xq))
    with torch.no_grad():
        ut = CDGSolve.apply(fq, torch.tensor(kstar, device="cuda"), cache)

    def loss(kap):
        with torch.no_grad():
            return float(((CDGSolve.apply(fq, torch.tensor(kap, device="cuda"), cache) - ut) ** 2).sum())
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
