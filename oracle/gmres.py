"""Right-preconditioned restarted GMRES(m) (Section 4: the outer Krylov method
of the paper, GMRES(50) with one V-cycle as right preconditioner; Section 5
stops it at a relative residual of 1e-8).

Test infrastructure only: the CUDA path never imports this module.

Textbook form (Saad, Iterative Methods for Sparse Linear Systems, 2nd ed.,
Section 9.3.2, right preconditioning): from r0 = b - A x0 and v1 = r0/||r0||,
the Arnoldi process on A M^{-1} with modified Gram-Schmidt builds V_{k+1} and
the (k+1) x k Hessenberg H_k; plane rotations reduce H_k to upper triangular
form and carry ||r0|| e1 along, so the last rotated entry |g_{k+1}| is the
residual norm of x_k = x0 + M^{-1} V_k y_k, y_k = argmin ||beta e1 - H_k y||.
A restart forms x_k explicitly, recomputes the true residual and begins a new
Arnoldi process.  Because the right preconditioner acts on the search space,
the residual that GMRES minimises is the unpreconditioned b - A x.

Conventions of this library (not fixed by the paper):
- iterations count Arnoldi steps (one preconditioner apply and one A apply each);
- hist[k] is |g_{k+1}|/||b|| after Arnoldi step k, hist[0] = ||r0||/||b||; at a
  restart the entry of the last step is replaced by the recomputed true
  residual;
- the process stops when hist[k] <= tol, or on a happy breakdown
  (h_{j+1,j} = 0: the Krylov space is invariant and x_k is exact).
"""
from __future__ import annotations

import numpy as np


def _givens(a: float, b: float):
    """c, s with [c s; -s c] [a; b] = [r; 0]."""
    if b == 0.0:
        return 1.0, 0.0
    r = np.hypot(a, b)
    return a / r, b / r


def gmres(A, b, precond=None, m=50, tol=1e-8, maxit=1000, x0=None):
    """Returns x, hist, iterations.  A and precond are callables or matrices."""
    Aop = A if callable(A) else (lambda v: A @ v)
    Mop = (lambda v: v) if precond is None else precond
    n = b.shape[0]
    bn = np.linalg.norm(b)
    x = np.zeros(n) if x0 is None else np.array(x0, dtype=float)
    if bn == 0.0:
        return np.zeros(n), [0.0], 0
    r = b - Aop(x)
    beta = np.linalg.norm(r)
    hist = [beta / bn]
    it = 0
    if hist[0] <= tol:
        return x, hist, 0
    while it < maxit:
        V = np.zeros((m + 1, n))
        H = np.zeros((m + 1, m))
        cs, sn = np.zeros(m), np.zeros(m)
        g = np.zeros(m + 1)
        g[0] = beta
        V[0] = r / beta
        k = 0
        converged = False
        while k < m and it < maxit:
            w = Aop(Mop(V[k]))
            for i in range(k + 1):          # modified Gram-Schmidt
                H[i, k] = w @ V[i]
                w = w - H[i, k] * V[i]
            H[k + 1, k] = np.linalg.norm(w)
            happy = H[k + 1, k] == 0.0
            if not happy:
                V[k + 1] = w / H[k + 1, k]
            for i in range(k):              # earlier rotations on the new column
                hi, hi1 = H[i, k], H[i + 1, k]
                H[i, k] = cs[i] * hi + sn[i] * hi1
                H[i + 1, k] = -sn[i] * hi + cs[i] * hi1
            cs[k], sn[k] = _givens(H[k, k], H[k + 1, k])
            H[k, k] = cs[k] * H[k, k] + sn[k] * H[k + 1, k]
            H[k + 1, k] = 0.0
            g[k + 1] = -sn[k] * g[k]
            g[k] = cs[k] * g[k]
            k += 1
            it += 1
            hist.append(abs(g[k]) / bn)
            if hist[-1] <= tol or happy:
                converged = True
                break
        # x_k = x0 + M^{-1} V_k y with H_k y = g (upper triangular, k x k)
        y = np.zeros(k)
        for i in range(k - 1, -1, -1):
            y[i] = (g[i] - H[i, i + 1:k] @ y[i + 1:k]) / H[i, i]
        x = x + Mop(V[:k].T @ y)
        r = b - Aop(x)
        beta = np.linalg.norm(r)
        hist[-1] = beta / bn
        if converged or hist[-1] <= tol:
            break
    return x, hist, it
