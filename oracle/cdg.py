r"""Level-0 CDG discretisation of Poisson's equation (Section 2).

R1 (sign): the paper prints Laplace(u) = f (eq. poisson) and +int f v in the
second weak equation (eq. poisson_weak); integrating div q = f against v gives
-int f v there, so the printed pair is inconsistent.  We solve -Laplace(u) = f,
for which A is symmetric positive definite and b carries +int f v.

Primal form (eq. primal_form), obtained by eliminating q_h with the CDG fluxes
(u-hat upwinded by the switch; q-hat = boundary gradient q^f of the q-side,
eq. edge_flux_interior; eq. cdg_fluxes on the boundary).  With [[u]] = u_a - u_b
on an interior face f whose q-side is a and u-side b, n the unit normal out of
a, and r_f(w) in [P_p(a)]^d the lifting int_a r.tau = int_f w tau.n:

  a(u,v) = sum_K kappa_K int_K grad u . grad v
         - sum_f kappa_a int_f ([[u]] dn v_a + [[v]] dn u_a)
         + sum_f kappa_a int_a r_f([[u]]) . r_f([[v]])
         + sum_{f in Gamma_D} kappa_K int_f (-u dn v - v dn u + C_D u v)
  b(v)   = int f v + sum_{Gamma_D} kappa_K int g_D (-dn v + C_D v) + sum_{Gamma_N} int g_N v

R5: on Dirichlet faces eq. edge_flux_boundary, read literally, gives
q^f = grad u_h, so no lifting term appears there.
R7 (per-element diffusion kappa, not in the paper): every term is weighted by
kappa of the element that owns it (volume: K; interior face: its q-side;
Dirichlet face: K), i.e. M is replaced by M / kappa_K in the flux form.
With orthonormal bases and flat faces, int_a r_f(w1).r_f(w2) =
sum_k (int_f w1 phi_k)(int_f w2 phi_k) over the basis phi of a.

Flux form pieces (eq. disc_grad, eq. flux_matrix_form): G with the paper's
sign, (G u)_{K,c,k} = int_K u div(tau) - int_{dK \ Gamma_D} u-hat tau.n for
tau = phi_k e_c; M the q-space mass matrix (block diagonal, Gram of the basis
times I_d, scaled by 1/kappa_K); D = -G^T; C = A + D M^{-1} G.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from .basis import Basis
from .mesh import Topology
from .quadrature import simplex_rule, map_simplex


class Level0:
    def __init__(self, mesh, p: int, gamma: float = 1e4, switch_kind: int = 0,
                 face_switch=None, enumeration=None, kappa=None, beta: float = 0.0, velocity=None):
        self.topo = t = Topology(mesh, switch_kind, face_switch, enumeration)
        # convection beta v . grad u (Section 5, convection-diffusion; R18: upwind DG)
        self.beta = float(beta)
        self.vel = np.zeros(t.d) if velocity is None else np.asarray(velocity, dtype=np.float64)[:t.d]
        self.p = p
        self.d = d = t.d
        self.bases = [Basis([t.simplex(K)], p) for K in range(t.ne)]
        self.np_ = len(self.bases[0].exps)
        self.C_D = gamma / t.h_avg
        self.kappa = np.ones(t.ne) if kappa is None else np.asarray(kappa, dtype=np.float64)
        self.vrule = simplex_rule(d, 2 * p)
        self.frule = simplex_rule(d - 1, 2 * p)

    def with_degree(self, q: int) -> "Level0":
        """The same discretisation (mesh, switch, C_D, kappa) at degree q: the
        rediscretised operators of the p-multigrid levels (Section 4.4)."""
        other = Level0.__new__(Level0)
        other.topo, other.p, other.d = self.topo, q, self.d
        other.bases = [Basis([self.topo.simplex(K)], q) for K in range(self.topo.ne)]
        other.np_ = len(other.bases[0].exps)
        other.C_D, other.kappa = self.C_D, self.kappa
        other.beta, other.vel = self.beta, self.vel
        other.vrule = simplex_rule(self.d, 2 * q)
        other.frule = simplex_rule(self.d - 1, 2 * q)
        return other

    # ---- quadrature points (the points at which the caller samples f, g_D, g_N)
    def volume_points(self, K):
        return map_simplex(self.topo.simplex(K), *self.vrule)

    def interior_face_points(self, f):
        return map_simplex(self.topo.if_verts[f], *self.frule)

    def boundary_face_points(self, bf):
        return map_simplex(self.topo.bf_verts[bf], *self.frule)

    def all_volume_points(self):
        return np.stack([self.volume_points(K)[0] for K in range(self.topo.ne)])

    def all_boundary_points(self):
        return np.stack([self.boundary_face_points(i)[0] for i in range(len(self.topo.boundary))])

    # ---- element-local pieces --------------------------------------------
    def volume_block(self, K):
        x, w = self.volume_points(K)
        g = self.bases[K].grad(x)
        return self.kappa[K] * np.einsum("q,qid,qjd->ij", w, g, g)

    def interior_face_blocks(self, f):
        """Blocks (aa, ab, ba, bb) of the interior-face terms of face f."""
        t = self.topo
        a, b = int(t.qside[f]), int(t.uside[f])
        Ka = t.interior[f][0]
        n = t.if_n[f] if a == Ka else -t.if_n[f]
        x, w = self.interior_face_points(f)
        pa = self.bases[a].eval(x)
        pb = self.bases[b].eval(x)
        dna = self.bases[a].grad(x) @ n
        k = self.kappa[a]
        aa = -(dna * w[:, None]).T @ pa - (pa * w[:, None]).T @ dna
        ab = (dna * w[:, None]).T @ pb
        ba = (pb * w[:, None]).T @ dna
        Qaa = (pa * w[:, None]).T @ pa
        Qab = (pa * w[:, None]).T @ pb
        aa = aa + Qaa.T @ Qaa
        ab = ab - Qaa.T @ Qab
        ba = ba - Qab.T @ Qaa
        bb = Qab.T @ Qab
        return a, b, k * aa, k * ab, k * ba, k * bb

    def dirichlet_block(self, bf):
        t = self.topo
        K, l, tag = t.boundary[bf]
        x, w = self.boundary_face_points(bf)
        n = t.bf_n[bf]
        ph = self.bases[K].eval(x)
        dn = self.bases[K].grad(x) @ n
        blk = (-(dn * w[:, None]).T @ ph - (ph * w[:, None]).T @ dn
               + self.C_D * (ph * w[:, None]).T @ ph)
        return K, self.kappa[K] * blk

    # ---- global operators --------------------------------------------------
    def blocks(self):
        """dict (row K, col J) -> n_p x n_p block of A_0."""
        t = self.topo
        B: dict[tuple[int, int], np.ndarray] = {}

        def add(i, j, m):
            if (i, j) in B:
                B[(i, j)] = B[(i, j)] + m
            else:
                B[(i, j)] = m.copy()
        for K in range(t.ne):
            add(K, K, self.volume_block(K))
        for f in range(len(t.interior)):
            a, b, aa, ab, ba, bb = self.interior_face_blocks(f)
            add(a, a, aa); add(a, b, ab); add(b, a, ba); add(b, b, bb)
        for bf, (K, l, tag) in enumerate(t.boundary):
            if tag == 0:
                K, blk = self.dirichlet_block(bf)
                add(K, K, blk)
        if self.beta != 0.0:
            for (i, j), m in self.convection_blocks().items():
                add(i, j, m)
        return B

    def convection_blocks(self):
        """R18: the convection term beta v . grad u of -div(kappa grad u) +
        beta v . grad u = f in upwind DG form (constant v, so div v = 0): on
        each element  -int_K u beta v.grad w  +  int_{dK} beta (v.n) u-hat w,
        u-hat the upwind trace (the element the flow leaves, v.n > 0 side), on
        the boundary u-hat = u_K at outflow and on Neumann faces, g_D at
        Dirichlet inflow (a right-hand-side term)."""
        t = self.topo
        bv = self.beta * self.vel
        B: dict[tuple[int, int], np.ndarray] = {}

        def add(i, j, m):
            B[(i, j)] = B[(i, j)] + m if (i, j) in B else m.copy()
        for K in range(t.ne):
            x, w = self.volume_points(K)
            ph = self.bases[K].eval(x)
            vg = self.bases[K].grad(x) @ bv                 # v . grad phi_i at the points
            add(K, K, -(vg * w[:, None]).T @ ph)
        for f, (K1, K2, _, _) in enumerate(t.interior):
            vn = float(bv @ t.if_n[f])                       # out of K1
            x, w = self.interior_face_points(f)
            p1, p2 = self.bases[K1].eval(x), self.bases[K2].eval(x)
            if vn > 0:      # flow leaves K1: u-hat = u_K1
                add(K1, K1, vn * (p1 * w[:, None]).T @ p1)
                add(K2, K1, -vn * (p2 * w[:, None]).T @ p1)
            elif vn < 0:    # flow leaves K2: u-hat = u_K2
                add(K1, K2, vn * (p1 * w[:, None]).T @ p2)
                add(K2, K2, -vn * (p2 * w[:, None]).T @ p2)
        for bf, (K, l, tag) in enumerate(t.boundary):
            vn = float(bv @ t.bf_n[bf])
            if vn > 0 or (tag == 1 and vn != 0):
                x, w = self.boundary_face_points(bf)
                ph = self.bases[K].eval(x)
                add(K, K, vn * (ph * w[:, None]).T @ ph)
        return B

    def matrix(self):
        return blocks_to_csr(self.blocks(), self.topo.ne, self.topo.ne, self.np_, self.np_)

    def gradient(self):
        """G (paper's sign, eq. disc_grad): [ne*d*n_p] x [ne*n_p]."""
        t = self.topo
        d, npb = self.d, self.np_
        B: dict[tuple[int, int], np.ndarray] = {}

        def add(i, j, m):
            B[(i, j)] = B[(i, j)] + m if (i, j) in B else m.copy()
        for K in range(t.ne):
            x, w = self.volume_points(K)
            ph = self.bases[K].eval(x)
            g = self.bases[K].grad(x)                      # [q, k, c]
            blk = np.zeros((d * npb, npb))
            for c in range(d):
                blk[c * npb:(c + 1) * npb] = np.einsum("q,qk,qj->kj", w, g[:, :, c], ph)
            add(K, K, blk)
        for f in range(len(t.interior)):
            a, b = int(t.qside[f]), int(t.uside[f])
            Ka = t.interior[f][0]
            na = t.if_n[f] if a == Ka else -t.if_n[f]
            x, w = self.interior_face_points(f)
            pa = self.bases[a].eval(x)
            pb = self.bases[b].eval(x)
            # q-side a takes u-hat = u_b; u-side b takes its own value
            blk_ab = np.zeros((d * npb, npb))
            blk_bb = np.zeros((d * npb, npb))
            for c in range(d):
                blk_ab[c * npb:(c + 1) * npb] = -na[c] * ((pa * w[:, None]).T @ pb)
                blk_bb[c * npb:(c + 1) * npb] = -(-na[c]) * ((pb * w[:, None]).T @ pb)
            add(a, b, blk_ab)
            add(b, b, blk_bb)
        for bf, (K, l, tag) in enumerate(t.boundary):
            if tag == 1:            # Neumann: u-hat = u_K
                x, w = self.boundary_face_points(bf)
                n = t.bf_n[bf]
                ph = self.bases[K].eval(x)
                blk = np.zeros((d * npb, npb))
                for c in range(d):
                    blk[c * npb:(c + 1) * npb] = -n[c] * ((ph * w[:, None]).T @ ph)
                add(K, K, blk)
        return blocks_to_csr(B, t.ne, t.ne, d * npb, npb)

    def mass_u(self):
        """Block-diagonal u-space mass matrix (Gram of each element basis)."""
        t = self.topo
        blocks = {}
        for K in range(t.ne):
            x, w = self.volume_points(K)
            ph = self.bases[K].eval(x)
            blocks[(K, K)] = (ph * w[:, None]).T @ ph
        return blocks_to_csr(blocks, t.ne, t.ne, self.np_, self.np_)

    def mass_q(self):
        """q-space mass matrix, scaled by 1/kappa_K (R7)."""
        t = self.topo
        blocks = {}
        for K in range(t.ne):
            x, w = self.volume_points(K)
            ph = self.bases[K].eval(x)
            m = (ph * w[:, None]).T @ ph
            blocks[(K, K)] = np.kron(np.eye(self.d), m) / self.kappa[K]
        return blocks_to_csr(blocks, t.ne, t.ne, self.d * self.np_, self.d * self.np_)

    def rhs(self, f_q, gD_q=None, gN_q=None):
        """b from f at the volume points [ne][nq] and g_D, g_N at the boundary
        face points [n_bfaces][nfq] (library boundary-face order)."""
        t = self.topo
        b = np.zeros((t.ne, self.np_))
        for K in range(t.ne):
            x, w = self.volume_points(K)
            b[K] += (self.bases[K].eval(x) * (w * f_q[K])[:, None]).sum(axis=0)
        for bf, (K, l, tag) in enumerate(t.boundary):
            x, w = self.boundary_face_points(bf)
            ph = self.bases[K].eval(x)
            if tag == 0 and gD_q is not None:
                dn = self.bases[K].grad(x) @ t.bf_n[bf]
                b[K] += self.kappa[K] * ((-dn + self.C_D * ph) * (w * gD_q[bf])[:, None]).sum(axis=0)
                vn = self.beta * float(self.vel @ t.bf_n[bf])
                if vn < 0:      # R18: Dirichlet inflow, u-hat = g_D
                    b[K] += -vn * (ph * (w * gD_q[bf])[:, None]).sum(axis=0)
            if tag == 1 and gN_q is not None:
                b[K] += (ph * (w * gN_q[bf])[:, None]).sum(axis=0)
        return b.ravel()


def blocks_to_csr(B, nr, nc, br, bc):
    rows, cols, vals = [], [], []
    for (i, j), m in B.items():
        ii, jj = np.meshgrid(np.arange(br) + i * br, np.arange(bc) + j * bc, indexing="ij")
        rows.append(ii.ravel()); cols.append(jj.ravel()); vals.append(m.ravel())
    if not rows:
        return sp.csr_matrix((nr * br, nc * bc))
    return sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                         shape=(nr * br, nc * bc))
