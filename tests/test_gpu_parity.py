"""GPU parity of every step of the solve phase against the FP64 oracle, called
through the C ABI (tree order on the device, the oracle's own numbering on the
host).

Two references per step.  (1) The library's own host operators (exported by
cdg_export_level, applied here in FP64 by scipy): this pins the kernels alone,
at 1e-13 for single applies.  (2) The oracle, which builds every operator
independently: agreement is limited by how far the two set-ups agree, `setup`
per case.  Both sides orthonormalise monomials through the Cholesky factor of
their Gram matrix (R2), whose condition number grows with the degree: the two
operators agree to ~1e-15 relative for triangles at p <= 3, 2e-13 at p = 4,
1e-11 at p = 5, 7e-11 at p = 6 and 1e-13 for tetrahedra at p = 3 (max-norm,
measured on these meshes).

Tolerances: single applies and transfers max(1e-13, setup); one smoothing step
additionally 4 eps max_K cond(D_K) ||omega D^-1 r|| / ||y||, because the
diagonal-block inverses are formed by two different factorisations that agree
only to cond(D_K) eps (cond(D_K) reaches 1e5 under C_D = 1e4/h_avg); the
coarsest solve (dense inverse plus one step of iterative refinement on the
device, LU in numpy) cond(A_n) eps; the V-cycle 1e-9; full solves 1e-10 relative
L2 (1e-10 + 100 setup where the two set-ups differ more) with iteration counts
within one of the oracle's."""
import numpy as np
import pytest
import scipy.sparse as sp

from synthetic import jittered_square, kuhn_cube, sin_source
from tests.gpu_common import OracleCase, rel

pytestmark = pytest.mark.gpu

EPS = 2.220446049250313e-16

# name: (mesh, options, setup agreement of library and oracle operators)
CASES = {
    "tri_p2_32": (lambda: jittered_square(32), dict(p=2, max_levels=4), 0.0),
    "tri_p3_16_mixed_bc": (lambda: jittered_square(16, neumann_axes=(0,)), dict(p=3, max_levels=4), 0.0),
    "tet_p2_4": (lambda: kuhn_cube(4), dict(p=2, max_levels=3), 0.0),
    "tet_p1_5": (lambda: kuhn_cube(5, seed=2), dict(p=1, max_levels=4, seed=3), 0.0),
    # block sizes n_p = 15, 21, 28 (triangles, p = 4, 5, 6) and n_p = 20 (tetrahedra, p = 3)
    "tri_p4_8": (lambda: jittered_square(8), dict(p=4, max_levels=3), 1e-12),
    "tri_p5_6_mixed_bc": (lambda: jittered_square(6, neumann_axes=(1,)), dict(p=5, max_levels=3), 1e-10),
    "tri_p6_6": (lambda: jittered_square(6), dict(p=6, max_levels=3), 5e-10),
    "tet_p3_3": (lambda: kuhn_cube(3), dict(p=3, max_levels=3), 1e-13),
}


def exported_operator(S, level):
    """A_l of the library's host set-up in tree order (scipy CSR) and the tree
    order itself (perm[k] = working index of tree row k)."""
    ex = S.export_level(level)
    npb = S.info["np_l"][level]
    n = len(ex["rowptr"]) - 1
    A = sp.bsr_matrix((ex["val"], ex["col"], ex["rowptr"]), shape=(n * npb, n * npb)).tocsr()
    return A, ex["perm"]


@pytest.fixture(scope="module", params=list(CASES))
def case(request):
    import torch
    from paper_2012_08024_gb300 import Solver
    mk, kw, setup = CASES[request.param]
    mesh = mk()
    S = Solver(mesh, **kw).bind()
    oc = OracleCase(mesh, kw["p"], kw["max_levels"], seed=kw.get("seed", 0))
    assert S.n_levels == oc.H.n_levels
    oc.setup = setup
    oc.kw = kw
    return S, oc, mesh


def _t(x):
    import torch
    return torch.tensor(np.ascontiguousarray(x), dtype=torch.float64, device="cuda")


def test_operator_apply_residual_smooth(case):
    import torch
    S, oc, _ = case
    rng = np.random.default_rng(1)
    tol = max(1e-13, oc.setup)
    for l in range(S.n_levels):
        A = oc.H.A[l]
        Ae, _ = exported_operator(S, l)
        n = A.shape[0]
        x = rng.standard_normal(n)
        b = rng.standard_normal(n)
        xt_np, bt_np = oc.to_tree(l, x), oc.to_tree(l, b)
        xt, bt = _t(xt_np), _t(bt_np)
        y = torch.empty_like(xt)
        S.apply(l, xt, y)
        torch.cuda.synchronize()
        ref = A @ x
        assert rel(y.cpu().numpy(), Ae @ xt_np) <= 1e-13
        assert rel(oc.to_work(l, y.cpu().numpy()), ref) <= tol
        S.residual(l, xt, bt, y)
        assert rel(y.cpu().numpy(), bt_np - Ae @ xt_np) <= 1e-13
        assert rel(oc.to_work(l, y.cpu().numpy()), b - ref) <= tol
        if l + 1 < S.n_levels:
            S.smooth(l, xt, bt, y)
            sm = oc.V.smooth(l, x, b)
            corr = sm - x
            npb = oc.npb
            Ad = A.tocsr()
            cond = max(np.linalg.cond(Ad[k * npb:(k + 1) * npb, k * npb:(k + 1) * npb].toarray())
                       for k in range(n // npb))
            tol_s = tol + 4 * EPS * cond * np.linalg.norm(corr) / np.linalg.norm(sm)
            assert rel(oc.to_work(l, y.cpu().numpy()), sm) <= tol_s


def test_restrict_prolong_coarse(case):
    import torch
    S, oc, _ = case
    rng = np.random.default_rng(2)
    tol = max(1e-13, oc.setup)
    for l in range(S.n_levels - 1):
        L = oc.H.L[l]
        r = rng.standard_normal(L.shape[0])
        bc = torch.empty(L.shape[1], dtype=torch.float64, device="cuda")
        S.restrict(l, _t(oc.to_tree(l, r)), bc)
        assert rel(oc.to_work(l + 1, bc.cpu().numpy()), L.T @ r) <= tol
        xc = rng.standard_normal(L.shape[1])
        x0 = rng.standard_normal(L.shape[0])
        xt = _t(oc.to_tree(l, x0))
        S.prolong(l, _t(oc.to_tree(l + 1, xc)), xt)
        assert rel(oc.to_work(l, xt.cpu().numpy()), x0 + L @ xc) <= tol
    # coarsest solve: against an LU solve of the library's own coarsest operator
    # (both backward stable: they agree to cond(A_n) eps) and of the oracle's
    Ae, _ = exported_operator(S, S.n_levels - 1)
    Ae = Ae.toarray()
    cond = np.linalg.cond(Ae)
    b = rng.standard_normal(Ae.shape[0])
    x = torch.empty(Ae.shape[0], dtype=torch.float64, device="cuda")
    S.coarse_solve(_t(b), x)
    assert rel(x.cpu().numpy(), np.linalg.solve(Ae, b)) <= 1e-14 + cond * EPS, (rel(x.cpu().numpy(),
                                                                                 np.linalg.solve(Ae, b)), cond)
    Ac = oc.H.A[-1].toarray()
    bw = oc.to_work(S.n_levels - 1, b)
    assert rel(oc.to_work(S.n_levels - 1, x.cpu().numpy()), np.linalg.solve(Ac, bw)) <= 1e-14 + cond * max(EPS, oc.setup)


def test_vcycle(case):
    import torch
    S, oc, _ = case
    r = np.random.default_rng(3).standard_normal(oc.H.A[0].shape[0])
    z = torch.empty(len(r), dtype=torch.float64, device="cuda")
    S.vcycle(_t(oc.to_tree(0, r)), z)
    assert rel(oc.to_work(0, z.cpu().numpy()), oc.V.apply(r)) <= 1e-9 + 100 * oc.setup


def test_fused_transfers_match_separate_kernels(case):
    """The V-cycle with the fused residual + restriction (+ first coarse smoothing
    step) and the prolongation carried by the coarse level's last sweep against
    the same cycle with separate kernels: the same arithmetic except the order
    of the per-agglomerate sums, whose rounding the coarsest solve amplifies by
    at most cond(A_n); and both against the oracle."""
    import torch
    from paper_2012_08024_gb300 import Solver
    S, oc, mesh = case
    S2 = Solver(mesh, fuse_transfers=3, **oc.kw).bind()
    Ae, _ = exported_operator(S, S.n_levels - 1)
    cond = np.linalg.cond(Ae.toarray())
    r = np.random.default_rng(31).standard_normal(oc.H.A[0].shape[0])
    z1 = torch.empty(len(r), dtype=torch.float64, device="cuda")
    z2 = torch.empty_like(z1)
    S.vcycle(_t(oc.to_tree(0, r)), z1)
    S2.vcycle(_t(oc.to_tree(0, r)), z2)
    d = rel(z1.cpu().numpy(), z2.cpu().numpy())
    assert d <= 1e-13 + 10 * cond * EPS, (d, cond)


def test_full_solve_matches_oracle(case):
    """Iteration counts within one of the oracle's.  Solutions: at equal
    iteration counts within 1e-10 relative L2 of the oracle's iterate; otherwise
    both within 1e-10 of the direct solution.  The GPU solution also solves the
    library's own level-0 system (exported operator, library right-hand side)
    to 1e-10."""
    import scipy.sparse.linalg as spl
    import torch
    from oracle.solver import pcg
    S, oc, mesh = case
    xq, xbq, btag = S.quadrature_points()
    fq = sin_source(xq)
    u, hist, it, rc = S.solve(_t(fq))
    assert rc == 0 and hist[-1] <= 1e-10, (rc, hist[-3:])
    b = oc.L0.rhs(fq)
    uo, ho, ito = pcg(oc.H.A[0], b, oc.V.apply, tol=1e-10)
    assert abs(it - ito) <= 1, (it, ito, hist[-3:], ho[-3:])
    ug = u.cpu().numpy().ravel()
    tol = 1e-10 + 100 * oc.setup
    if it == ito:
        assert rel(ug, uo) <= tol, (it, ito, rel(ug, uo))
    else:
        ud = spl.spsolve(oc.H.A[0].tocsc(), b)
        assert rel(ug, ud) <= tol and rel(uo, ud) <= 1e-10, (it, ito, rel(ug, ud), rel(uo, ud))
    # the library's own system, in tree order
    A0, perm = exported_operator(S, 0)
    bl = S.rhs(_t(fq)).cpu().numpy()
    ut = spl.spsolve(A0.tocsc(), bl[perm].ravel())
    assert rel(u.cpu().numpy()[perm].ravel(), ut) <= 1e-10
    # the true residual of the GPU solution, by the oracle's operator
    assert np.linalg.norm(b - oc.H.A[0] @ ug) <= (2e-10 + 100 * oc.setup) * np.linalg.norm(b)
    # host-pointer path gives the same answer
    uh, hh, ith, rch = S.solve_host(fq)
    assert ith == it and rel(uh, u.cpu().numpy()) <= 1e-14


def test_rhs_matches_oracle(case):
    import torch
    S, oc, mesh = case
    xq, xbq, btag = S.quadrature_points()
    rng = np.random.default_rng(4)
    fq = rng.standard_normal(xq.shape[:2])
    gD = rng.standard_normal(xbq.shape[:2])
    gN = rng.standard_normal(xbq.shape[:2])
    b = S.rhs(_t(fq), _t(gD), _t(gN))
    assert rel(b.cpu().numpy(), oc.L0.rhs(fq, gD, gN)) <= max(1e-13, oc.setup)


def test_edge_cases():
    import torch
    from paper_2012_08024_gb300 import Solver
    from oracle.cdg import Level0
    # single level: the V-cycle is the dense solve, CG converges in one step
    m = jittered_square(3)
    S = Solver(m, p=1, max_levels=1).bind()
    xq, _, _ = S.quadrature_points()
    u, hist, it, rc = S.solve(_t(sin_source(xq)))
    assert rc == 0 and it <= 2
    L0 = Level0(m, 1)
    ud = np.linalg.solve(L0.matrix().toarray(), L0.rhs(sin_source(xq)))
    assert rel(u.cpu().numpy(), ud) <= 1e-10
    # zero right-hand side: zero solution, no iteration
    u0, h0, it0, rc0 = S.solve(_t(np.zeros(xq.shape[:2])))
    assert it0 == 0 and not u0.abs().max().item()
    # two elements
    from synthetic.meshes import Mesh
    two = Mesh(2, np.array([[0., 0.], [1., 0.], [1., 1.], [0., 1.]]), np.array([[0, 1, 2], [0, 2, 3]]),
               np.zeros((0, 2), dtype=np.int64), np.zeros(0, dtype=np.int32))
    S2 = Solver(two, p=2, max_levels=3).bind()
    assert S2.n_levels == 2
    xq2, _, _ = S2.quadrature_points()
    u2, h2, it2, rc2 = S2.solve(_t(sin_source(xq2)))
    L2 = Level0(two, 2)
    ud2 = np.linalg.solve(L2.matrix().toarray(), L2.rhs(sin_source(xq2)))
    assert rc2 == 0 and rel(u2.cpu().numpy(), ud2) <= 1e-10
    # maxit exhaustion is reported, outputs written
    S3 = Solver(jittered_square(8), p=2, max_levels=2, maxit=2).bind()
    xq3, _, _ = S3.quadrature_points()
    u3, h3, it3, rc3 = S3.solve(_t(sin_source(xq3)))
    assert rc3 == 3 and it3 == 2 and np.isfinite(u3.cpu().numpy()).all()


def test_binding_checks_device_tensors():
    """A wrong dtype, a short buffer or a non-contiguous view is refused by the
    binding before the call; the handle stays usable."""
    import torch
    from paper_2012_08024_gb300 import Solver
    S = Solver(jittered_square(6), p=2, max_levels=2).bind()
    n = S.info["n_l"][0] * S.np_
    x = torch.zeros(n, dtype=torch.float64, device="cuda")
    y = torch.empty_like(x)
    with pytest.raises(ValueError, match="dtype"):
        S.apply(0, x.float(), y)
    with pytest.raises(ValueError, match="at least"):
        S.apply(0, x[: n - 1], y)
    with pytest.raises(ValueError, match="contiguous"):
        S.apply(0, torch.zeros(2 * n, dtype=torch.float64, device="cuda")[::2], y)
    S.apply(0, x, y)
    torch.cuda.synchronize()
    assert not y.abs().max().item()


def test_unaligned_caller_vectors(case):
    """Caller vectors that are not 16-byte aligned take the kernel without
    vector loads; results agree with the aligned call."""
    import torch
    S, oc, _ = case
    n = oc.H.A[0].shape[0]
    big = torch.tensor(np.random.default_rng(7).standard_normal(n + 1), dtype=torch.float64, device="cuda")
    xa = big[:n].clone()
    xu = big[1:]
    xu.copy_(xa)
    ya, yu = torch.empty_like(xa), torch.empty(n + 1, dtype=torch.float64, device="cuda")[1:]
    S.apply(0, xa, ya)
    S.apply(0, xu, yu)
    torch.cuda.synchronize()
    assert rel(yu.cpu().numpy(), ya.cpu().numpy()) <= 1e-14


def test_fp32_operator_copy():
    """cdg_apply_f32: the FP32 copy of A_l that the FP32 V-cycle uses, against the
    oracle's FP64 operator (FP32 rounding of blocks, vector and sums)."""
    import torch
    from paper_2012_08024_gb300 import Solver
    from oracle.cdg import Level0
    from oracle.hierarchy import MGHierarchy
    mesh = jittered_square(16)
    S = Solver(mesh, p=3, max_levels=3, precision="fp32").bind()
    H = MGHierarchy(Level0(mesh, 3), max_levels=3)
    order = H.tree_order()
    rng = np.random.default_rng(5)
    for l in range(S.n_levels - 1):
        n = H.A[l].shape[0]
        x = rng.standard_normal(n)
        xt = x.reshape(-1, 10)[order[l]].ravel()
        y = torch.empty(n, dtype=torch.float32, device="cuda")
        S.apply_f32(l, torch.tensor(xt, dtype=torch.float32, device="cuda"), y)
        yw = np.empty((len(order[l]), 10))
        yw[order[l]] = y.cpu().numpy().astype(np.float64).reshape(-1, 10)
        ref = H.A[l] @ x
        assert rel(yw.ravel(), ref) <= 1e-5, (l, rel(yw.ravel(), ref))


def test_solve_stops_at_maxit_with_the_oracle_history():
    """The CG loop runs as one graph whose condition the device clears; at maxit
    it stops with CDG_ENOCONV, and the recorded residual history equals the
    oracle's PCG history entry by entry."""
    from paper_2012_08024_gb300 import Solver
    from oracle.solver import pcg
    mesh = jittered_square(12)
    S = Solver(mesh, p=2, max_levels=3, maxit=5, tol=1e-14).bind()
    oc = OracleCase(mesh, 2, 3)
    xq, _, _ = S.quadrature_points()
    fq = sin_source(xq)
    assert not S.solve_graph()
    u, hist, it, rc = S.solve(_t(fq))
    assert S.solve_graph()          # the loop ran as one graph launch, not the host-driven fallback
    assert rc == 3 and it == 5 and len(hist) == 6
    uo, ho, ito = pcg(oc.H.A[0], oc.L0.rhs(fq), oc.V.apply, tol=1e-14, maxit=5)
    assert ito == 5
    assert np.all(np.abs(hist - np.asarray(ho)) <= 1e-8 * np.asarray(ho))
    assert rel(u.cpu().numpy().ravel(), uo) <= 1e-10


@pytest.mark.parametrize("krylov,precision", [("cg", "fp64"), ("cg", "fp32"), ("gmres", "fp64")])
def test_single_graph_and_host_driven_loops_are_identical(krylov, precision):
    """The one-graph solve (conditional WHILE node) and the host-driven loop run
    the same kernels in the same order: identical iterates, histories and counts."""
    from paper_2012_08024_gb300 import Solver
    mesh = jittered_square(14)
    kw = dict(p=2, max_levels=3, precision=precision, krylov=krylov)
    if krylov == "gmres":
        kw.update(nu_pre=0, nu_post=3, restart=10, tol=1e-10)
    out = []
    for single in (True, False):
        S = Solver(mesh, single_graph=single, **kw).bind()
        u, hist, it, rc = S.solve(_t(sin_source(S.quadrature_points()[0])))
        assert rc == 0 and S.solve_graph() == single
        out.append((u.cpu().numpy(), hist, it))
    assert out[0][2] == out[1][2]
    assert np.array_equal(out[0][1], out[1][1])
    assert np.array_equal(out[0][0], out[1][0])


def test_tetrahedral_flux_coarsening_needs_more_iterations():
    """Beyond the paper (2D only): on the Kuhn-split cube the flux-coarsened
    hierarchy needs clearly more PCG iterations than primal coarsening (oracle,
    8^3 x 6, p = 1, V(1,1): 120 against 80), the reverse of the 2D result."""
    from paper_2012_08024_gb300 import Solver
    mesh = kuhn_cube(12)
    its = {}
    for coarsen in ("flux", "primal"):
        S = Solver(mesh, p=1, max_levels=6, coarsen=coarsen, maxit=1000).bind()
        u, hist, it, rc = S.solve(_t(sin_source(S.quadrature_points()[0])))
        assert rc == 0
        its[coarsen] = it
    print("12^3 x 6, p = 1, V(1,1):", its)
    assert its["flux"] >= 1.25 * its["primal"], its
