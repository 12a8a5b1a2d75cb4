"""Pins of the oracle's p-multigrid front end (Section 4.4; reading R17:
degrees p, p-1, ..., 1 on the fine mesh with the CDG operator rediscretised at
each degree, then the agglomeration hierarchy of the p = 1 discretisation).

* Nested bases: the orthonormal graded bases of degree q-1 are the leading
  functions of the degree-q basis on the same element, so the prolongation
  integral L_K = int_K phi_K psi_K^T is the truncation [I; 0].
* The rediscretised degree-q operator is the Section 2 operator at that
  degree, pinned by the operator pins (symmetry, SPD, polynomial
  reproduction); here: its leading block equals the degree-q operator only up
  to the lifting term, which is degree dependent (so the levels are not
  Galerkin products), while the volume and face terms nest exactly.
* The agglomeration part is exactly the p = 1 hierarchy.
* With nu1 = nu2 the V-cycle is symmetric and positive definite, PCG with it
  reaches the dense solution, and it needs fewer iterations than the
  agglomeration-only V-cycle at the same degree.
"""
import numpy as np
import pytest

from oracle.cdg import Level0
from oracle.hierarchy import MGHierarchy
from oracle.solver import VCycle, pcg
from synthetic import jittered_square, kuhn_cube, sin_source


@pytest.fixture(scope="module", params=["tri_p3", "tet_p2"])
def case(request):
    if request.param == "tri_p3":
        L0 = Level0(jittered_square(6, neumann_axes=(0,)), 3)
    else:
        L0 = Level0(kuhn_cube(2), 2)
    return L0, MGHierarchy(L0, max_levels=4, seed=1, pmg=True)


def test_levels_and_nested_transfers(case):
    L0, H = case
    assert H.deg[:H.n_plevels + 1] == list(range(L0.p, 0, -1))
    assert all(q == 1 for q in H.deg[H.n_plevels:])
    for l in range(H.n_plevels):
        for LK in H.Lblk[l]:
            assert LK.shape == (H.nps[l], H.nps[l + 1])
            assert np.abs(LK - np.eye(*LK.shape)).max() <= 1e-12


def test_agglomeration_part_is_the_p1_hierarchy(case):
    L0, H = case
    H1 = MGHierarchy(L0.with_degree(1), max_levels=4, seed=1)
    assert H.n_levels == H.n_plevels + H1.n_levels
    for l in range(H1.n_levels):
        a, b = H.A[H.n_plevels + l].toarray(), H1.A[l].toarray()
        assert np.abs(a - b).max() <= 1e-13 * np.abs(b).max()


def test_volume_and_face_terms_nest_but_lifting_does_not(case):
    """A_q restricted to degree q-1 differs from A_{q-1} (the lifting into
    [P_q]^d is larger than into [P_{q-1}]^d) but by a positive semidefinite
    amount: a larger lifting space gives at least the same lifting energy."""
    L0, H = case
    for l in range(H.n_plevels):
        n1 = H.nps[l + 1]
        A, Ac = H.A[l].toarray(), H.A[l + 1].toarray()
        npf = H.nps[l]
        idx = np.concatenate([np.arange(K * npf, K * npf + n1) for K in range(A.shape[0] // npf)])
        lead = A[np.ix_(idx, idx)]
        diff = lead - Ac
        assert np.abs(diff).max() > 1e-8 * np.abs(Ac).max()
        assert np.linalg.eigvalsh((diff + diff.T) / 2).min() >= -1e-9 * np.abs(Ac).max()


def test_vcycle_symmetric_and_solve(case):
    L0, H = case
    V = VCycle(H.A, H.L, H.nps, 1, 1)
    n = H.A[0].shape[0]
    B = np.stack([V.apply(e) for e in np.eye(n)], axis=1)
    assert np.abs(B - B.T).max() <= 1e-11 * np.abs(B).max()
    assert np.linalg.eigvalsh((B + B.T) / 2).min() > 0
    b = L0.rhs(sin_source(L0.all_volume_points()))
    x, hist, it = pcg(H.A[0], b, V.apply, tol=1e-12)
    xd = np.linalg.solve(H.A[0].toarray(), b)
    assert np.linalg.norm(x - xd) <= 1e-10 * np.linalg.norm(xd)


def test_fewer_iterations_than_agglomeration_only():
    L0 = Level0(jittered_square(12), 3)
    b = L0.rhs(sin_source(L0.all_volume_points()))
    its = []
    for pmg in (False, True):
        H = MGHierarchy(L0, max_levels=16, pmg=pmg)
        V = VCycle(H.A, H.L, H.nps, 1, 1)
        its.append(pcg(H.A[0], b, V.apply, tol=1e-10)[2])
    assert its[1] < 0.8 * its[0], its      # measured 70 -> 46


def test_p1_pmg_is_plain_hierarchy():
    L0 = Level0(jittered_square(5), 1)
    Ha, Hb = MGHierarchy(L0, max_levels=3, pmg=True), MGHierarchy(L0, max_levels=3)
    assert Ha.n_plevels == 0 and Ha.n_levels == Hb.n_levels
    for a, b in zip(Ha.A, Hb.A):
        assert np.abs((a - b).toarray()).max() == 0.0
