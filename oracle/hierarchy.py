"""Multigrid hierarchy: bases on agglomerates, transfers, flux coarsening
(Sections 3.3-4.1).

* Basis on every agglomerate: Basis(R2) over its fine sub-simplices; its
  integrals are sums over those sub-elements (Section 3.3).
* Prolongation (Section 3.4): injection, L_K = int_K phi_K psi_A^T for a
  level-l element K inside the level-(l+1) agglomerate A (exact: psi_A|K is in
  P_p(K)).  Restriction: M^{l+1} R = (M^l L)^T.
* Flux coarsening (Section 4.1): [[M, G], [D, C]]_{l+1} = diag(R_q, R) [[M, G],
  [D, C]]_l diag(L_q, L), with L_q = L acting on every component of q (the
  q-space is [P_p]^d on the same elements) and R_q its restriction; then
  A_{l+1} = C_{l+1} - D_{l+1} M_{l+1}^{-1} G_{l+1}.
  R13: C_l is used exactly, second-neighbour blocks included (the paper's
  "implicitly inferred" read as C_l = A_l + D_l M_l^{-1} G_l, formed here).
  R13' (option compact_c): the second-neighbour blocks of C_l that lie across
  two different agglomerates are dropped before coarsening.
  Primal coarsening (Section 3.5, option primal): A_{l+1} = R A_l L.
* p-multigrid front end (Section 4.4, option pmg; reading R17): for p > 1
  the hierarchy first lowers the degree on the fine mesh, p, p-1, ..., 1
  (standard p-multigrid: each element is its own coarse element and the coarse
  space is P_{q-1} on the same element), with the CDG operator rediscretised
  at every degree, and then continues with the agglomeration hierarchy of the
  p = 1 discretisation.  The prolongation between degrees is the same
  integral L_K = int_K phi_K psi_K^T (nested orthonormal bases make it the
  truncation [I; 0]).  Flux coarsening between degrees is not used: it makes
  the degree p-1 operator indefinite (lambda_min = -1858 on a 5 x 5 square at
  p = 3).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from .agglomerate import Hierarchy
from .basis import Basis
from .cdg import Level0, blocks_to_csr
from .quadrature import simplex_rule, map_simplex


def block_diag_inverse(Mcsr, nb, bs):
    blocks = {}
    Md = Mcsr.toarray() if nb * bs <= 4000 else None
    for K in range(nb):
        sl = slice(K * bs, (K + 1) * bs)
        blk = Md[sl, sl] if Md is not None else Mcsr[sl, sl].toarray()
        blocks[(K, K)] = np.linalg.inv(blk)
    return blocks_to_csr(blocks, nb, nb, bs, bs)


class MGHierarchy:
    def __init__(self, lvl0: Level0, max_levels: int, seed: int = 0, coarsen: str = "flux", pmg: bool = False):
        t = lvl0.topo
        self.lvl0 = lvl0
        self.p, self.d, self.np_ = lvl0.p, lvl0.d, lvl0.np_
        if pmg and lvl0.p > 1:
            self._build_pmg(lvl0, max_levels, seed, coarsen)
            return
        self.agg = Hierarchy([list(map(int, t.elem[K])) for K in range(t.ne)], t.nbrs, max_levels, seed)
        # levels: n_p degree-lowering levels on the fine mesh, then the agglomeration levels
        self.n_plevels = 0
        hdeg = self.p
        self.deg = [hdeg] * self.agg.n_levels
        self.n_levels = len(self.deg)
        self.nps = [_n_basis(self.d, q) for q in self.deg]
        self.members = [self.agg.members[h] for h in range(self.agg.n_levels)]
        self.parent = [self.agg.parent[h] for h in range(self.agg.n_levels - 1)]
        simplex = [t.simplex(K) for K in range(t.ne)]
        self.bases = [lvl0.bases]
        for l in range(1, self.n_levels):
            self.bases.append([Basis([simplex[m] for m in mem], self.deg[l]) for mem in self.members[l]])
        rp, rw = simplex_rule(self.d, 2 * self.p)
        # prolongation blocks L_K (n_p(l) x n_p(l+1)) and sparse L per level
        self.Lblk, self.L, self.Mu = [], [], []
        for l in range(self.n_levels):
            nl, npl = len(self.members[l]), self.nps[l]
            mb = {}
            for K in range(nl):
                g = np.zeros((npl, npl))
                for m in self.members[l][K]:
                    x, w = map_simplex(simplex[m], rp, rw)
                    ph = self.bases[l][K].eval(x)
                    g += (ph * w[:, None]).T @ ph
                mb[(K, K)] = g
            self.Mu.append(blocks_to_csr(mb, nl, nl, npl, npl))
        for l in range(self.n_levels - 1):
            par = self.parent[l]
            nl, nc = len(par), len(self.members[l + 1])
            npf, npc = self.nps[l], self.nps[l + 1]
            blocks, B = [], {}
            for K in range(nl):
                A = par[K]
                LK = np.zeros((npf, npc))
                for m in self.members[l][K]:
                    x, w = map_simplex(simplex[m], rp, rw)
                    LK += (self.bases[l][K].eval(x) * w[:, None]).T @ self.bases[l + 1][A].eval(x)
                blocks.append(LK)
                B[(K, A)] = LK
            self.Lblk.append(blocks)
            self.L.append(blocks_to_csr(B, nl, nc, npf, npc))
        # level-0 flux form
        A0 = lvl0.matrix()
        G0 = lvl0.gradient()
        M0 = lvl0.mass_q()
        D0 = -G0.T.tocsr()
        M0inv = block_diag_inverse(M0, t.ne, self.d * self.np_)
        C0 = (A0 + D0 @ M0inv @ G0).tocsr()
        self.A, self.G, self.M, self.D, self.C = [A0], [G0], [M0], [D0], [C0]
        for l in range(self.n_levels - 1):
            L = self.L[l]
            npf, npc = self.nps[l], self.nps[l + 1]
            nc = L.shape[1] // npc
            R = self.restriction(l)
            Lq = _q_prolongation(L, self.d, npf, npc)
            Rq = _q_prolongation(R.T.tocsr(), self.d, npf, npc).T.tocsr()
            if coarsen == "primal":
                Ac = (R @ self.A[l] @ L).tocsr()
                self.A.append(Ac); self.G.append(None); self.M.append(None); self.D.append(None); self.C.append(None)
                continue
            Cl = self.C[l]
            if coarsen == "compact_c":
                Cl = _drop_cross_agglomerate_2hop(Cl, self.parent[l], npf, self.A[l])
            Mc = (Rq @ self.M[l] @ Lq).tocsr()
            Gc = (Rq @ self.G[l] @ L).tocsr()
            Dc = (R @ self.D[l] @ Lq).tocsr()
            Cc = (R @ Cl @ L).tocsr()
            Mcinv = block_diag_inverse(Mc, nc, self.d * npc)
            Ac = (Cc - Dc @ Mcinv @ Gc).tocsr()
            self.A.append(Ac); self.G.append(Gc); self.M.append(Mc); self.D.append(Dc); self.C.append(Cc)

    def _build_pmg(self, lvl0, max_levels, seed, coarsen):
        """R17: levels of degree p, p-1, ..., 2 on the fine mesh (rediscretised),
        then the whole hierarchy of the degree-1 discretisation."""
        t = lvl0.topo
        H1 = MGHierarchy(lvl0.with_degree(1), max_levels, seed, coarsen)
        self.h1 = H1
        self.agg = H1.agg
        fine_levels = [lvl0] + [lvl0.with_degree(q) for q in range(self.p - 1, 1, -1)]
        self.n_plevels = len(fine_levels)
        self.deg = [f.p for f in fine_levels] + H1.deg
        self.nps = [f.np_ for f in fine_levels] + H1.nps
        self.n_levels = len(self.deg)
        fine = [[K] for K in range(t.ne)]
        self.members = [fine] * self.n_plevels + H1.members
        self.parent = [list(range(t.ne))] * self.n_plevels + H1.parent
        self.bases = [f.bases for f in fine_levels] + H1.bases
        self.Mu = []
        for f in fine_levels:
            mb = {}
            for K in range(t.ne):
                x, w = map_simplex(t.simplex(K), *f.vrule)
                ph = f.bases[K].eval(x)
                mb[(K, K)] = (ph * w[:, None]).T @ ph
            self.Mu.append(blocks_to_csr(mb, t.ne, t.ne, f.np_, f.np_))
        self.Mu += H1.Mu
        # prolongation between consecutive degrees: L_K = int_K phi_K (degree q) psi_K^T (degree q-1)
        rp, rw = simplex_rule(self.d, 2 * self.p)
        self.Lblk, self.L = [], []
        coarse_fine = fine_levels[1:] + [H1.lvl0]
        for f, c in zip(fine_levels, coarse_fine):
            blocks, B = [], {}
            for K in range(t.ne):
                x, w = map_simplex(t.simplex(K), rp, rw)
                LK = (f.bases[K].eval(x) * w[:, None]).T @ c.bases[K].eval(x)
                blocks.append(LK)
                B[(K, K)] = LK
            self.Lblk.append(blocks)
            self.L.append(blocks_to_csr(B, t.ne, t.ne, f.np_, c.np_))
        self.Lblk += H1.Lblk
        self.L += H1.L
        self.A = [f.matrix() for f in fine_levels] + H1.A
        none = [None] * self.n_plevels
        self.G, self.M, self.D, self.C = none + H1.G, none + H1.M, none + H1.D, none + H1.C

    def restriction(self, l):
        npf, npc = self.nps[l], self.nps[l + 1]
        nc = self.L[l].shape[1] // npc
        return (block_diag_inverse(self.Mu[l + 1], nc, npc) @ (self.Mu[l] @ self.L[l]).T).tocsr()

    def tree_order(self):
        """Tree numbering of every level: the degree-lowering levels share the
        numbering of the fine agglomeration level."""
        t = self.agg.tree_order()
        return [t[0]] * self.n_plevels + list(t)


def _n_basis(d, p):
    """dim P_p in d variables = C(p + d, d)."""
    from math import comb
    return comb(p + d, d)


def _q_prolongation(L, d, npf, npc):
    """L_q: the u-space prolongation (fine n_p npf, coarse npc) applied to each
    of the d components of a q-vector stored as [element][component][basis]."""
    Lc = L.tocoo()
    rows, cols, vals = [], [], []
    for c in range(d):
        rows.append((Lc.row // npf) * d * npf + c * npf + Lc.row % npf)
        cols.append((Lc.col // npc) * d * npc + c * npc + Lc.col % npc)
        vals.append(Lc.data)
    return sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                         shape=(L.shape[0] * d, L.shape[1] * d))


def _drop_cross_agglomerate_2hop(C, par, npb, A):
    """R13': zero the blocks of C that are not blocks of A (second neighbours)
    and whose two elements lie in different agglomerates of level l+1."""
    Cc = C.tocoo()
    Ap = set(zip(*[x // npb for x in A.nonzero()]))
    keep = np.array([((r // npb, c // npb) in Ap) or par[r // npb] == par[c // npb]
                     for r, c in zip(Cc.row, Cc.col)], dtype=bool)
    return sp.csr_matrix((Cc.data[keep], (Cc.row[keep], Cc.col[keep])), shape=C.shape)
