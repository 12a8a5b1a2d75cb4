"""V-cycle preconditioned CG (Section 4.3, Algorithm 3; Section 5 set-up).

R14: the printed V-cycle listing is garbled (it never smooths level 0, returns
x^(0) unchanged and loops "i = n_pre" on the way up).  We read it as the
standard V(nu1, nu2) cycle: on levels 0..n-1, starting from x = 0, nu1 damped
block-Jacobi steps x += alpha D^{-1} (b - A x) (alpha = 2/3, D = the diagonal
blocks of A_l), restrict the residual, solve level n directly, prolongate and
add the correction, nu2 smoothing steps.  With nu1 = nu2 it is symmetric.
R15: the outer Krylov method is CG (A is SPD, Section 4) with the V-cycle as
preconditioner, x0 = 0 (Section 5), stopped when ||r_k||/||b|| <= tol on the
recurrence residual; iterations count the A_0 applies after the initial
residual.  The flexible form beta = (r_new, z_new - z_old)/(r_old, z_old)
(Polak-Ribiere) is available for preconditioners that are not exactly
symmetric (lower precision V-cycles).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp


class VCycle:
    def __init__(self, A: list, L: list, npb, nu1: int = 1, nu2: int = 1,
                 omega: float = 2.0 / 3.0, R: list | None = None):
        """npb: basis functions per element, one value for every level or a
        list with one value per level (p-multigrid levels)."""
        self.A, self.L = A, L
        self.npbs = list(npb) if hasattr(npb, "__len__") else [npb] * len(A)
        self.npb = self.npbs[0]
        self.R = R if R is not None else [Li.T.tocsr() for Li in L]
        self.nu1, self.nu2, self.omega = nu1, nu2, omega
        self.Dinv = []
        for Al, npl in zip(A[:-1], self.npbs):
            n = Al.shape[0] // npl
            blocks = []
            for K in range(n):
                sl = slice(K * npl, (K + 1) * npl)
                blocks.append(np.linalg.inv(Al[sl, sl].toarray()))
            self.Dinv.append(sp.block_diag(blocks, format="csr"))
        self.coarse = np.linalg.inv(A[-1].toarray())
        self.Acoarse = A[-1].toarray()

    def smooth(self, l, x, b):
        return x + self.omega * (self.Dinv[l] @ (b - self.A[l] @ x))

    def apply(self, b, l=0):
        if l == len(self.A) - 1:
            return np.linalg.solve(self.Acoarse, b)
        x = np.zeros_like(b)
        for _ in range(self.nu1):
            x = self.smooth(l, x, b)
        r = b - self.A[l] @ x
        xc = self.apply(self.R[l] @ r, l + 1)
        x = x + self.L[l] @ xc
        for _ in range(self.nu2):
            x = self.smooth(l, x, b)
        return x


def pcg(A, b, precond, tol=1e-10, maxit=500, x0=None, flexible=False):
    """Returns x, residual history ||r_k||/||b||, iterations."""
    bn = np.linalg.norm(b)
    x = np.zeros_like(b) if x0 is None else x0.copy()
    if bn == 0.0:
        return np.zeros_like(b), [0.0], 0
    r = b - A @ x
    hist = [np.linalg.norm(r) / bn]
    if hist[0] <= tol:
        return x, hist, 0
    z = precond(r)
    p = z.copy()
    rho = r @ z
    it = 0
    while it < maxit:
        q = A @ p
        alpha = rho / (p @ q)
        x = x + alpha * p
        r = r - alpha * q
        it += 1
        hist.append(np.linalg.norm(r) / bn)
        if hist[-1] <= tol:
            break
        z_new = precond(r)
        rho_new = r @ z_new
        beta = (rho_new - r @ z) / rho if flexible else rho_new / rho
        z = z_new
        p = z + beta * p
        rho = rho_new
    return x, hist, it
