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
    def __init__(self, lvl0: Level0, max_levels: int, seed: int = 0, coarsen: str = "flux"):
        t = lvl0.topo
        self.lvl0 = lvl0
        self.p, self.d, self.np_ = lvl0.p, lvl0.d, lvl0.np_
        self.agg = Hierarchy([list(map(int, t.elem[K])) for K in range(t.ne)], t.nbrs, max_levels, seed)
        self.n_levels = self.agg.n_levels
        simplex = [t.simplex(K) for K in range(t.ne)]
        # bases on every level (level 0: one simplex per element)
        self.bases = [lvl0.bases]
        for l in range(1, self.n_levels):
            self.bases.append([Basis([simplex[m] for m in mem], self.p) for mem in self.agg.members[l]])
        rp, rw = simplex_rule(self.d, 2 * self.p)
        # prolongation blocks L_K and sparse L per level
        self.Lblk, self.L, self.Mu = [], [], []
        for l in range(self.n_levels):
            nl = len(self.agg.members[l])
            mb = {}
            for K in range(nl):
                g = np.zeros((self.np_, self.np_))
                for m in self.agg.members[l][K]:
                    x, w = map_simplex(simplex[m], rp, rw)
                    ph = self.bases[l][K].eval(x)
                    g += (ph * w[:, None]).T @ ph
                mb[(K, K)] = g
            self.Mu.append(blocks_to_csr(mb, nl, nl, self.np_, self.np_))
        for l in range(self.n_levels - 1):
            par = self.agg.parent[l]
            nl, nc = len(par), len(self.agg.members[l + 1])
            blocks, B = [], {}
            for K in range(nl):
                A = par[K]
                LK = np.zeros((self.np_, self.np_))
                for m in self.agg.members[l][K]:
                    x, w = map_simplex(simplex[m], rp, rw)
                    LK += (self.bases[l][K].eval(x) * w[:, None]).T @ self.bases[l + 1][A].eval(x)
                blocks.append(LK)
                B[(K, A)] = LK
            self.Lblk.append(blocks)
            self.L.append(blocks_to_csr(B, nl, nc, self.np_, self.np_))
        # level-0 flux form
        A0 = lvl0.matrix()
        G0 = lvl0.gradient()
        M0 = lvl0.mass_q()
        D0 = -G0.T.tocsr()
        M0inv = block_diag_inverse(M0, t.ne, self.d * self.np_)
        C0 = (A0 + D0 @ M0inv @ G0).tocsr()
        self.A, self.G, self.M, self.D, self.C = [A0], [G0], [M0], [D0], [C0]
        eye_d = sp.identity(self.d, format="csr")
        for l in range(self.n_levels - 1):
            L = self.L[l]
            nc = L.shape[1] // self.np_
            R = self.restriction(l)
            Lq = _q_prolongation(L, self.d, self.np_)
            Rq = _q_prolongation(R.T.tocsr(), self.d, self.np_).T.tocsr()
            if coarsen == "primal":
                Ac = (R @ self.A[l] @ L).tocsr()
                self.A.append(Ac); self.G.append(None); self.M.append(None); self.D.append(None); self.C.append(None)
                continue
            Cl = self.C[l]
            if coarsen == "compact_c":
                Cl = _drop_cross_agglomerate_2hop(Cl, self.agg, l, self.np_, self.A[l])
            Mc = (Rq @ self.M[l] @ Lq).tocsr()
            Gc = (Rq @ self.G[l] @ L).tocsr()
            Dc = (R @ self.D[l] @ Lq).tocsr()
            Cc = (R @ Cl @ L).tocsr()
            Mcinv = block_diag_inverse(Mc, nc, self.d * self.np_)
            Ac = (Cc - Dc @ Mcinv @ Gc).tocsr()
            self.A.append(Ac); self.G.append(Gc); self.M.append(Mc); self.D.append(Dc); self.C.append(Cc)

    def restriction(self, l):
        nc = self.L[l].shape[1] // self.np_
        return (block_diag_inverse(self.Mu[l + 1], nc, self.np_) @ (self.Mu[l] @ self.L[l]).T).tocsr()


def _q_prolongation(L, d, npb):
    """L_q: the u-space prolongation applied to each of the d components of a
    q-vector stored as [element][component][basis]."""
    Lc = L.tocoo()
    rows, cols, vals = [], [], []
    for c in range(d):
        rows.append((Lc.row // npb) * d * npb + c * npb + Lc.row % npb)
        cols.append((Lc.col // npb) * d * npb + c * npb + Lc.col % npb)
        vals.append(Lc.data)
    return sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                         shape=(L.shape[0] * d, L.shape[1] * d))


def _drop_cross_agglomerate_2hop(C, agg, l, npb, A):
    """R13': zero the blocks of C that are not blocks of A (second neighbours)
    and whose two elements lie in different agglomerates of level l+1."""
    par = agg.parent[l]
    Cc = C.tocoo()
    Ap = set(zip(*[x // npb for x in A.nonzero()]))
    keep = np.array([((r // npb, c // npb) in Ap) or par[r // npb] == par[c // npb]
                     for r, c in zip(Cc.row, Cc.col)], dtype=bool)
    return sp.csr_matrix((Cc.data[keep], (Cc.row[keep], Cc.col[keep])), shape=C.shape)
