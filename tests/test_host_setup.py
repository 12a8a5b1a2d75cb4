"""Host logic of the library against the oracle (CPU only, no device calls):
the library's C++ set-up and the oracle share no code, so agreement pins both.

* Algorithm 2 agglomeration: parents of every level bit-identical;
* tree numbering bit-identical (children of every agglomerate contiguous);
* A_l on every level (flux coarsening, Section 4.1) within 1e-12 relative;
* transfer blocks L_K (Section 3.4) within 1e-12, and upper triangular up to
  rounding for every supported degree;
* quadrature points (R3) and boundary-face order / tags identical;
* errors: degenerate element and missing Dirichlet boundary are rejected.
"""
import numpy as np
import pytest

from oracle.cdg import Level0
from oracle.hierarchy import MGHierarchy
from synthetic import jittered_square, kuhn_cube
from synthetic.meshes import Mesh


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2012_08024_gb300 import build
    build.build()


def _dense(ex, n, npb):
    A = np.zeros((n * npb, n * npb))
    for k in range(n):
        for b in range(ex["rowptr"][k], ex["rowptr"][k + 1]):
            j = ex["col"][b]
            A[k * npb:(k + 1) * npb, j * npb:(j + 1) * npb] = ex["val"][b]
    return A


CASES = [
    ("tri_p2_mixed", lambda: jittered_square(6, neumann_axes=(0,)), dict(p=2, max_levels=4)),
    ("tri_p3", lambda: jittered_square(8), dict(p=3, max_levels=3)),
    ("tet_p1", lambda: kuhn_cube(2), dict(p=1, max_levels=3)),
    ("tet_p2_seed", lambda: kuhn_cube(2, seed=4), dict(p=2, max_levels=3, seed=11)),
    ("tri_natural", lambda: jittered_square(5), dict(p=1, max_levels=3, switch_kind=1)),
    ("tri_p4", lambda: jittered_square(4), dict(p=4, max_levels=3)),
    ("tri_p6", lambda: jittered_square(3), dict(p=6, max_levels=2)),
    ("tet_p3", lambda: kuhn_cube(2), dict(p=3, max_levels=3)),
    ("tri_kappa", lambda: jittered_square(5), dict(p=2, max_levels=3,
                                                  kappa=np.exp(np.random.default_rng(1).standard_normal(50)))),
    ("tri_p3_pmg", lambda: jittered_square(8, neumann_axes=(1,)), dict(p=3, max_levels=3, pmg=True)),
    ("tet_p2_pmg", lambda: kuhn_cube(2), dict(p=2, max_levels=3, pmg=True)),
    ("tri_p2_pmg_kappa", lambda: jittered_square(5), dict(p=2, max_levels=3, pmg=True,
                                                         kappa=np.exp(np.random.default_rng(2).standard_normal(50)))),
    ("tri_p2_convection", lambda: jittered_square(6, neumann_axes=(0,)),
     dict(p=2, max_levels=3, beta=10.0, velocity=(1.0, 0.3), krylov="gmres")),
    ("tet_p1_convection", lambda: kuhn_cube(2), dict(p=1, max_levels=3, beta=3.0, velocity=(0.2, -1.0, 0.5),
                                                     krylov="gmres")),
    ("tri_p3_pmg_convection", lambda: jittered_square(6), dict(p=3, max_levels=3, pmg=True, beta=50.0,
                                                               velocity=(1.0, 0.0), krylov="gmres")),
]


@pytest.mark.parametrize("name,mk,kw", CASES, ids=[c[0] for c in CASES])
def test_library_setup_matches_oracle(name, mk, kw):
    from paper_2012_08024_gb300 import Solver
    mesh = mk()
    S = Solver(mesh, **kw)
    okw = dict(p=kw["p"], switch_kind=kw.get("switch_kind", 0), kappa=kw.get("kappa"),
               beta=kw.get("beta", 0.0), velocity=kw.get("velocity"))
    L0 = Level0(mesh, **okw)
    H = MGHierarchy(L0, max_levels=kw["max_levels"], seed=kw.get("seed", 0), pmg=kw.get("pmg", False))
    assert S.n_levels == H.n_levels
    assert S.info["np_l"] == H.nps and S.info["n_plevels"] == H.n_plevels
    order = H.tree_order()
    # both sides orthonormalise monomials through the Cholesky factor of their Gram
    # matrix, whose condition number grows with the degree: the two roundings
    # agree to 1e-12 up to p = 4 and to ~1e-10 at p = 6
    rtol = 1e-12 if kw["p"] <= 4 else 1e-9
    for l in range(H.n_levels - 1):
        assert list(S.export_agglomeration(l)) == list(H.parent[l])
    for l in range(H.n_levels):
        npb = H.nps[l]
        ex = S.export_level(l)
        assert list(ex["perm"]) == list(order[l])
        n = len(order[l])
        P = np.zeros((n * npb, n * npb))
        for k, w in enumerate(order[l]):
            P[k * npb:(k + 1) * npb, w * npb:(w + 1) * npb] = np.eye(npb)
        Aor = P @ H.A[l].toarray() @ P.T
        Alib = _dense(ex, n, npb)
        assert np.abs(Alib - Aor).max() <= rtol * np.abs(Aor).max()
        if l + 1 < H.n_levels:
            Lor = np.array([H.Lblk[l][w] for w in order[l]])
            assert np.abs(ex["L"] - Lor).max() <= rtol
            pos = {w: k for k, w in enumerate(order[l + 1])}
            assert list(ex["parent"]) == [pos[H.parent[l][w]] for w in order[l]]
    xq, xbq, btag = S.quadrature_points()
    assert np.abs(xq - L0.all_volume_points()).max() < 1e-14
    assert np.abs(xbq - L0.all_boundary_points()).max() < 1e-14
    assert list(btag) == [t for (_, _, t) in L0.topo.boundary]
    assert abs(S.info["C_D"] - L0.C_D) <= 1e-12 * L0.C_D


@pytest.mark.parametrize("dim,p", [(2, 1), (2, 2), (2, 3), (2, 4), (2, 5), (2, 6), (3, 1), (3, 2), (3, 3)])
def test_transfer_blocks_upper_triangular(dim, p):
    """Below the diagonal only rounding remains; it grows with the degree (the
    Gram matrices of the monomials worsen) to ~7e-11 of a block at p = 6."""
    from paper_2012_08024_gb300 import Solver
    mesh = jittered_square(12, seed=7) if dim == 2 else kuhn_cube(3, seed=7)
    S = Solver(mesh, p=p, max_levels=4)
    for l in range(S.n_levels - 1):
        L = S.export_level(l)["L"]
        low = np.abs(np.tril(L, -1)).max(axis=(1, 2))
        assert np.all(low <= 1e-9 * np.abs(L).max(axis=(1, 2))), (l, low.max())


def test_agglomeration_bit_exact_larger_mesh():
    from paper_2012_08024_gb300 import Solver
    from oracle.agglomerate import Hierarchy
    from oracle.mesh import Topology
    mesh = jittered_square(40, seed=3)
    S = Solver(mesh, p=1, max_levels=6, seed=5)
    t = Topology(mesh)
    Ho = Hierarchy([list(map(int, e)) for e in mesh.elem], t.nbrs, 6, 5)
    for l in range(Ho.n_levels - 1):
        assert list(S.export_agglomeration(l)) == Ho.parent[l]


@pytest.mark.parametrize("shape", ["square128", "cube16"])
@pytest.mark.parametrize("seed", [0, 1, 2, 3, 4])
def test_agglomeration_bit_exact_config_sizes(shape, seed):
    """Algorithm 2 applied recursively (7 levels) on a 128 x 128 jittered square
    (32,768 triangles) and a 16^3 x 6 Kuhn cube (24,576 tetrahedra), five mesh
    and tie-break seeds each: every parent of every level and the tree numbering
    of the library equal the oracle's."""
    from paper_2012_08024_gb300 import Solver
    from oracle.agglomerate import Hierarchy
    from oracle.mesh import Topology
    mesh = jittered_square(128, seed=seed) if shape == "square128" else kuhn_cube(16, seed=seed)
    S = Solver(mesh, p=1, max_levels=7, seed=17 * seed + 1)
    t = Topology(mesh)
    Ho = Hierarchy([list(map(int, e)) for e in mesh.elem], t.nbrs, 7, 17 * seed + 1)
    assert S.n_levels == Ho.n_levels == 7
    for l in range(Ho.n_levels - 1):
        assert list(S.export_agglomeration(l)) == Ho.parent[l], l
    order = Ho.tree_order()
    for l in range(Ho.n_levels):
        assert list(S.export_level(l)["perm"]) == list(order[l]), l


def test_errors_are_reported():
    from paper_2012_08024_gb300 import CdgError, Solver
    m = jittered_square(2)
    bad = Mesh(2, m.xyz.copy(), m.elem.copy(), m.bface, m.btag)
    bad.elem[0] = [0, 1, 2]        # collinear vertices 0, 1, 2 on y = 0
    with pytest.raises(CdgError) as e:
        Solver(bad, p=1)
    assert e.value.code == 2
    allneu = Mesh(2, m.xyz, m.elem, m.bface, np.ones(len(m.btag), dtype=np.int32))
    with pytest.raises(CdgError) as e:
        Solver(allneu, p=1)
    assert e.value.code == 2 and "Dirichlet" in str(e.value)
    with pytest.raises(CdgError) as e:
        Solver(m, p=0)
    assert e.value.code == 1


def test_malformed_meshes_are_rejected():
    """Inputs that would otherwise be read out of range or silently ignored."""
    from paper_2012_08024_gb300 import CdgError, Solver
    m = jittered_square(2)
    i32, i64 = np.int32, np.int64
    bad = {
        "empty mesh": Mesh(2, m.xyz, np.zeros((0, 3), dtype=i64), np.zeros((0, 2), dtype=i64), np.zeros(0, dtype=i32)),
        "out of range": Mesh(2, m.xyz, np.vstack([m.elem[:-1], [[0, 1, 999]]]), m.bface, m.btag),
        "btag must be 0": Mesh(2, m.xyz, m.elem, m.bface, np.full(len(m.btag), 5, dtype=i32)),
        "not a boundary face": Mesh(2, m.xyz, m.elem, np.vstack([m.bface, [[0, 4]]]).astype(i64),
                                    np.append(m.btag, 0).astype(i32)),
        "listed twice": Mesh(2, m.xyz, m.elem, np.vstack([m.bface, m.bface[:1]]).astype(i64),
                             np.append(m.btag, m.btag[0]).astype(i32)),
    }
    xyz = m.xyz.copy()
    xyz[3, 0] = np.nan
    bad["must be finite"] = Mesh(2, xyz, m.elem, m.bface, m.btag)
    for msg, mesh in bad.items():
        with pytest.raises(CdgError) as e:
            Solver(mesh, p=1)
        assert e.value.code == 1 and msg in str(e.value), (msg, str(e.value))


def test_malformed_options_are_rejected():
    from paper_2012_08024_gb300 import CdgError, Solver
    m = jittered_square(3)
    ne = m.n_elements
    bad = [
        (dict(gamma=np.inf), "bad omega"),
        (dict(omega=np.nan), "bad omega"),
        (dict(coarsen="flux", switch_kind=2), "are 0 or 1"),
        (dict(switch_kind=1, enumeration=np.zeros(ne, dtype=np.int64)), "distinct"),
    ]
    for kw, msg in bad:
        with pytest.raises(CdgError) as e:
            Solver(m, p=1, **kw)
        assert e.value.code == 1 and msg in str(e.value), (kw, str(e.value))
    S = Solver(m, p=1)
    nif = S.info["n_interior_faces"]
    with pytest.raises(CdgError) as e:
        Solver(m, p=1, face_switch=np.zeros(nif, dtype=np.int8))
    assert e.value.code == 1 and "+1 or -1" in str(e.value)
    Solver(m, p=1, face_switch=np.where(np.arange(nif) % 2 == 0, 1, -1).astype(np.int8))
    with pytest.raises(CdgError) as e:
        Solver(kuhn_cube(2), p=4)
    assert e.value.code == 1 and "p <= 3" in str(e.value)
    # cdg_solve_multi exists for n_p = 3, 4, 6, 10 only
    for mesh, p in ((m, 4), (kuhn_cube(2), 3)):
        with pytest.raises(CdgError) as e:
            Solver(mesh, p=p, nrhs=8, precision="fp32")
        assert e.value.code == 1 and "n_p = 3, 4, 6 or 10" in str(e.value)
    Solver(m, p=3, nrhs=8, precision="fp32")


def test_convection_options_are_checked():
    from paper_2012_08024_gb300 import CdgError, Solver
    m = jittered_square(4)
    for kw in (dict(beta=1.0), dict(beta=1.0, krylov="gmres", nrhs=4), dict(beta=float("nan"), krylov="gmres")):
        with pytest.raises(CdgError) as e:
            Solver(m, p=1, velocity=(1.0, 0.0), **kw)
        assert e.value.code == 1


def test_gmres_options_and_device_bytes():
    """GMRES(m) (Section 4) is an option of cdg_solve: checked at creation, and
    its Krylov storage (m + 1 basis and m preconditioned vectors) is part of
    the device buffer."""
    from paper_2012_08024_gb300 import CdgError, Solver
    m = jittered_square(6)
    cg = Solver(m, p=2)
    gm = Solver(m, p=2, nu_pre=0, nu_post=3, krylov="gmres", restart=10)
    ndofs = cg.info["n_dofs"]
    extra = gm.info["device_bytes"] - cg.info["device_bytes"]
    assert 21 * ndofs * 8 <= extra <= 21 * (ndofs + 32) * 8 + 64 * 1024
    for kw in (dict(krylov="gmres", restart=0), dict(krylov="gmres", restart=513)):
        with pytest.raises(CdgError) as e:
            Solver(m, p=1, **kw)
        assert e.value.code == 1 and "restart" in str(e.value)
