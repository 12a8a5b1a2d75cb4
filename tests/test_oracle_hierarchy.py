"""Pins of the oracle's transfers and coarse operators (Sections 3.3-4.1).

* M_l = I on every level (orthonormal bases) and R = L^T; sum_K L_K^T L_K = I.
* Coarse A_l symmetric positive definite.
* Independent route: G_l equals the LDG gradient assembled directly on the
  agglomerated mesh of level l (its own volume and boundary-face integrals,
  inherited fine faces and switch), and A_l = P_l^T C_0 P_l + G_l^T G_l with
  P_l[K, E] = int_K phi_K psi_E^T the direct level-l -> level-0 injection.
* Primal coarsening (A_{l+1} = R A_l L) differs from flux coarsening.
* Every transfer block L_K is upper triangular: with bases graded by degree in
  (x - c)/h (a scalar h) and orthonormalised in that order, the parent's
  function j restricted to a child lies in the span of the child's functions
  0..j (an affine map with isotropic scaling keeps each monomial's leading term).
"""
import numpy as np
import pytest
import scipy.sparse as sp

from oracle.cdg import Level0
from oracle.hierarchy import MGHierarchy
from oracle.quadrature import simplex_rule, map_simplex
from synthetic import jittered_square, kuhn_cube


@pytest.fixture(scope="module", params=["tri", "tet", "tri_pmg", "tet_pmg"])
def hier(request):
    if request.param == "tri":
        return MGHierarchy(Level0(jittered_square(6, neumann_axes=(0,)), 2), max_levels=4, seed=3)
    if request.param == "tet":
        return MGHierarchy(Level0(kuhn_cube(2), 1), max_levels=4, seed=3)
    if request.param == "tri_pmg":    # p = 3, 2, 1 on the fine mesh, then agglomeration at p = 1
        return MGHierarchy(Level0(jittered_square(5, neumann_axes=(0,)), 3), max_levels=3, seed=3, pmg=True)
    return MGHierarchy(Level0(kuhn_cube(2), 2), max_levels=3, seed=3, pmg=True)


def test_mass_identity_and_transfer(hier):
    for l in range(hier.n_levels):
        assert np.abs(hier.Mu[l] - sp.identity(hier.Mu[l].shape[0])).max() < 1e-12
        if hier.M[l] is not None:
            assert np.abs(hier.M[l] - sp.identity(hier.M[l].shape[0])).max() < 1e-12
    for l in range(hier.n_levels - 1):
        L = hier.L[l]
        assert np.abs(L.T @ L - sp.identity(L.shape[1])).max() < 1e-12
        assert np.abs(hier.restriction(l) - L.T).max() < 1e-12


def test_transfer_blocks_upper_triangular(hier):
    for l in range(hier.n_levels - 1):
        for LK in hier.Lblk[l]:
            assert np.abs(np.tril(LK, -1)).max(initial=0.0) <= 1e-12 * np.abs(LK).max()


def test_coarse_operators_symmetric_positive(hier):
    for A in hier.A:
        Ad = A.toarray()
        assert np.abs(Ad - Ad.T).max() <= 1e-12 * np.abs(Ad).max()
        assert np.linalg.eigvalsh(Ad).min() > 0


def _direct_ldg_gradient(hier, l):
    """LDG gradient (paper's sign, eq. disc_grad) assembled on the level-l
    agglomerates: volume integrals over their sub-simplices, face integrals
    over fine faces between different agglomerates (switch inherited) and
    fine Neumann faces; faces inside an agglomerate drop out."""
    L0 = hier.lvl0
    t = L0.topo
    d, npb = hier.d, hier.nps[l]
    owner = np.zeros(t.ne, dtype=int)
    for E, mem in enumerate(hier.members[l]):
        owner[mem] = E
    B = hier.bases[l]
    nE = len(B)
    G = np.zeros((nE * d * npb, nE * npb))
    rp, rw = L0.vrule
    for K in range(t.ne):
        E = owner[K]
        x, w = map_simplex(t.simplex(K), rp, rw)
        ph, g = B[E].eval(x), B[E].grad(x)
        for c in range(d):
            G[(E * d + c) * npb:(E * d + c + 1) * npb, E * npb:(E + 1) * npb] += \
                np.einsum("q,qk,qj->kj", w, g[:, :, c], ph)
    for f in range(len(t.interior)):
        a, b = int(t.qside[f]), int(t.uside[f])
        Ea, Eb = owner[a], owner[b]
        if Ea == Eb:
            continue
        na = t.if_n[f] if a == t.interior[f][0] else -t.if_n[f]
        x, w = L0.interior_face_points(f)
        pa, pb = B[Ea].eval(x), B[Eb].eval(x)
        for c in range(d):
            G[(Ea * d + c) * npb:(Ea * d + c + 1) * npb, Eb * npb:(Eb + 1) * npb] -= na[c] * (pa * w[:, None]).T @ pb
            G[(Eb * d + c) * npb:(Eb * d + c + 1) * npb, Eb * npb:(Eb + 1) * npb] += na[c] * (pb * w[:, None]).T @ pb
    for bf, (K, lf, tag) in enumerate(t.boundary):
        if tag != 1:
            continue
        E = owner[K]
        x, w = L0.boundary_face_points(bf)
        ph = B[E].eval(x)
        for c in range(d):
            G[(E * d + c) * npb:(E * d + c + 1) * npb, E * npb:(E + 1) * npb] -= t.bf_n[bf][c] * (ph * w[:, None]).T @ ph
    return G


def _direct_injection(hier, l):
    L0 = hier.lvl0
    t = L0.topo
    npb, npl = hier.np_, hier.nps[l]
    P = np.zeros((t.ne * npb, len(hier.bases[l]) * npl))
    rp, rw = L0.vrule
    for E, mem in enumerate(hier.members[l]):
        for K in mem:
            x, w = map_simplex(t.simplex(K), rp, rw)
            P[K * npb:(K + 1) * npb, E * npl:(E + 1) * npl] = \
                (L0.bases[K].eval(x) * w[:, None]).T @ hier.bases[l][E].eval(x)
    return P


def test_coarse_operator_independent_route(hier):
    if hier.n_plevels:
        pytest.skip("p-multigrid levels are rediscretised; their agglomeration part is the p = 1 hierarchy")
    C0 = hier.C[0].toarray()
    for l in range(1, hier.n_levels):
        Gd = _direct_ldg_gradient(hier, l)
        Gc = hier.G[l].toarray()
        assert np.abs(Gc - Gd).max() <= 1e-12 * np.abs(Gd).max()
        P = _direct_injection(hier, l)
        Ad = P.T @ C0 @ P + Gd.T @ Gd
        Ac = hier.A[l].toarray()
        assert np.abs(Ac - Ad).max() <= 1e-11 * np.abs(Ad).max()


def test_primal_differs_from_flux():
    L0 = Level0(jittered_square(6), 1)
    Hf = MGHierarchy(L0, max_levels=2)
    Hp = MGHierarchy(L0, max_levels=2, coarsen="primal")
    Ap, Af = Hp.A[1].toarray(), Hf.A[1].toarray()
    assert np.abs(Ap - Af).max() > 1e-5 * np.abs(Af).max()
    # primal is the Galerkin product
    R = Hf.L[0].T
    assert np.abs(Ap - (R @ Hf.A[0] @ Hf.L[0]).toarray()).max() < 1e-12 * np.abs(Ap).max()


def test_harmonic_polynomial_annihilated_away_from_dirichlet():
    # P = x^2 - y^2 + 3xy is harmonic: A_l P_l vanishes on agglomerates whose
    # fine elements are all at least two fine faces away from Gamma_D
    L0 = Level0(jittered_square(10), 2)
    H = MGHierarchy(L0, max_levels=3)
    t = L0.topo
    near = set(K for (K, lf, tag) in t.boundary if tag == 0)
    near |= set(nb for K in list(near) for nb in t.nbrs[K])
    near |= set(nb for K in list(near) for nb in t.nbrs[K])
    P = lambda x: x[..., 0] ** 2 - x[..., 1] ** 2 + 3 * x[..., 0] * x[..., 1]
    for l in range(H.n_levels):
        rp, rw = L0.vrule
        vals = []
        for E, mem in enumerate(H.agg.members[l]):
            v = np.zeros(H.np_)
            for K in mem:
                x, w = map_simplex(t.simplex(K), rp, rw)
                v += (H.bases[l][E].eval(x) * (w * P(x))[:, None]).sum(0)
            vals.append(v)
        y = (H.A[l] @ np.concatenate(vals)).reshape(-1, H.np_)
        scale = np.abs(H.A[l]).max() * np.abs(np.concatenate(vals)).max()
        far = [E for E, mem in enumerate(H.agg.members[l]) if not (set(mem) & near)]
        if l == 0:
            assert far
        for E in far:
            # coarse rows: the correction term only vanishes where the whole
            # second coarse neighbourhood is away from Gamma_D
            nb2 = {E} | set(H.agg.nbrs[l][E])
            nb2 |= {n2 for n1 in list(nb2) for n2 in H.agg.nbrs[l][n1]}
            if any(set(H.agg.members[l][e]) & near for e in nb2):
                continue
            assert np.abs(y[E]).max() <= 1e-10 * scale
