"""Adjoint of the solve u = A_0(kappa)^{-1} b(f, kappa) (differentiation of
eq. primal_form; the paper itself has no adjoint).

R7 makes A_0 and b linear in kappa with every term owned by one element: the
volume term by its element, an interior face by its q-side, a Dirichlet face
(operator and data term) by its element.  Hence, for a loss L(u) and the
adjoint state A_0^T lambda = dL/du,
    dL/dkappa_K = lambda^T (db/dkappa_K - dA_0/dkappa_K u),
    dL/df(x_q) on element K = sum_i w_q phi_i(x_q) lambda_K[i].
"""
from __future__ import annotations

import numpy as np

from .cdg import Level0


def kappa_gradient(L0: Level0, lam: np.ndarray, u: np.ndarray, gD_q=None) -> np.ndarray:
    t = L0.topo
    npb = L0.np_
    U = u.reshape(t.ne, npb)
    Lm = lam.reshape(t.ne, npb)
    g = np.zeros(t.ne)
    for K in range(t.ne):
        g[K] -= Lm[K] @ (L0.volume_block(K) / L0.kappa[K]) @ U[K]
    for f in range(len(t.interior)):
        a, b, aa, ab, ba, bb = L0.interior_face_blocks(f)
        s = Lm[a] @ aa @ U[a] + Lm[a] @ ab @ U[b] + Lm[b] @ ba @ U[a] + Lm[b] @ bb @ U[b]
        g[a] -= s / L0.kappa[a]
    for bf, (K, l, tag) in enumerate(t.boundary):
        if tag != 0:
            continue
        K, blk = L0.dirichlet_block(bf)
        g[K] -= Lm[K] @ blk @ U[K] / L0.kappa[K]
        if gD_q is not None:
            x, w = L0.boundary_face_points(bf)
            ph = L0.bases[K].eval(x)
            dn = L0.bases[K].grad(x) @ t.bf_n[bf]
            db = ((-dn + L0.C_D * ph) * (w * gD_q[bf])[:, None]).sum(axis=0)
            g[K] += Lm[K] @ db
    return g


def rhs_gradient(L0: Level0, lam: np.ndarray) -> np.ndarray:
    t = L0.topo
    Lm = lam.reshape(t.ne, L0.np_)
    out = np.zeros((t.ne, len(L0.vrule[1])))
    for K in range(t.ne):
        x, w = L0.volume_points(K)
        out[K] = w * (L0.bases[K].eval(x) @ Lm[K])
    return out
