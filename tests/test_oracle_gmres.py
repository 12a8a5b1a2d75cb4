"""Pins of the oracle's right-preconditioned restarted GMRES(m) (the outer
Krylov method of Section 4 / Section 5).

What fixes GMRES independently of its own code: after k Arnoldi steps from x0
its iterate minimises ||b - A x|| over x0 + M^{-1} K_k(A M^{-1}, r0), which a
least-squares solve on the explicit Krylov basis computes by brute force; with
m >= n it terminates at the exact solution; GMRES(1) with M = I is the
minimal-residual iteration x += (r.Ar)/(Ar.Ar) r.
"""
import numpy as np
import pytest

from oracle.cdg import Level0
from oracle.gmres import gmres
from oracle.hierarchy import MGHierarchy
from oracle.solver import VCycle
from synthetic import jittered_square, sin_source


def _system(n=12, seed=0, symmetric=False):
    rng = np.random.default_rng(seed)
    B = rng.standard_normal((n, n)) / np.sqrt(n)
    # well conditioned, so that the explicit Krylov basis of the brute force stays accurate
    A = 3.0 * np.eye(n) + ((B + B.T) / 2 if symmetric else B)
    P = np.eye(n) + 0.3 * rng.standard_normal((n, n)) / np.sqrt(n)   # M^{-1}
    b = rng.standard_normal(n)
    x0 = rng.standard_normal(n)
    return A, P, b, x0


def _min_residual(A, P, b, x0, k):
    """min ||b - A x|| over x in x0 + P span{r0, (AP) r0, ..., (AP)^{k-1} r0}."""
    r0 = b - A @ x0
    K = [r0]
    for _ in range(k - 1):
        K.append(A @ (P @ K[-1]))
    K = np.stack(K, axis=1)
    y, *_ = np.linalg.lstsq(A @ P @ K, r0, rcond=None)
    return np.linalg.norm(r0 - A @ P @ K @ y)


@pytest.mark.parametrize("symmetric", [False, True])
def test_residual_is_krylov_minimum(symmetric):
    A, P, b, x0 = _system(symmetric=symmetric)
    bn = np.linalg.norm(b)
    K = 7
    x, hist, it = gmres(A, b, lambda v: P @ v, m=20, tol=0.0, maxit=K, x0=x0)
    assert it == K and len(hist) == K + 1
    assert hist[0] == pytest.approx(np.linalg.norm(b - A @ x0) / bn, rel=1e-14)
    for k in range(1, K + 1):
        assert hist[k] == pytest.approx(_min_residual(A, P, b, x0, k) / bn, rel=1e-9, abs=1e-14)
    # the last entry is the recomputed true residual of the returned x
    assert hist[-1] == pytest.approx(np.linalg.norm(b - A @ x) / bn, rel=1e-12)


def test_finite_termination_and_direct_solve():
    A, P, b, _ = _system(n=10, seed=3)
    x, hist, it = gmres(A, b, lambda v: P @ v, m=10, tol=1e-13, maxit=10)
    xd = np.linalg.solve(A, b)
    assert it <= 10
    assert np.linalg.norm(x - xd) <= 1e-11 * np.linalg.norm(xd)


def test_gmres1_is_minimal_residual_iteration():
    A, _, b, x0 = _system(n=15, seed=5, symmetric=True)
    steps = 6
    x, hist, it = gmres(A, b, None, m=1, tol=0.0, maxit=steps, x0=x0)
    xm = x0.copy()
    for _ in range(steps):
        r = b - A @ xm
        Ar = A @ r
        xm = xm + (r @ Ar) / (Ar @ Ar) * r
    assert it == steps
    assert np.linalg.norm(x - xm) <= 1e-12 * np.linalg.norm(xm)
    assert hist[-1] == pytest.approx(np.linalg.norm(b - A @ xm) / np.linalg.norm(b), rel=1e-10)


def test_restarts_decrease_and_converge():
    A, P, b, _ = _system(n=40, seed=7)
    x, hist, it = gmres(A, b, lambda v: P @ v, m=4, tol=1e-12, maxit=400)
    assert hist[-1] <= 1e-12
    assert np.linalg.norm(b - A @ x) <= 2e-12 * np.linalg.norm(b)
    # within a cycle the residual never grows (minimisation over nested spaces)
    for c in range(0, len(hist) - 1, 4):
        seg = hist[c:c + 5]
        assert all(seg[i + 1] <= seg[i] * (1 + 1e-12) for i in range(len(seg) - 1))


def test_zero_rhs_and_exact_guess():
    A, P, b, _ = _system(n=8, seed=9)
    x, hist, it = gmres(A, np.zeros(8), lambda v: P @ v)
    assert it == 0 and not x.any()
    xd = np.linalg.solve(A, b)
    x, hist, it = gmres(A, b, lambda v: P @ v, x0=xd, tol=1e-8)
    assert it == 0


@pytest.mark.parametrize("coarsen", ["flux", "primal"])
def test_vcycle_right_preconditioned_cdg(coarsen):
    """The paper's setting on a small CDG problem: GMRES(50), V(0,3), tol 1e-8."""
    L0 = Level0(jittered_square(8, neumann_axes=(0,)), 1)
    H = MGHierarchy(L0, max_levels=10, coarsen=coarsen)
    V = VCycle(H.A, H.L, L0.np_, 0, 3)
    b = L0.rhs(sin_source(L0.all_volume_points()))
    x, hist, it = gmres(H.A[0], b, V.apply, m=50, tol=1e-8)
    xd = np.linalg.solve(H.A[0].toarray(), b)
    assert hist[-1] <= 1e-8 and it < 50
    assert np.linalg.norm(H.A[0] @ x - b) <= 1e-8 * np.linalg.norm(b)
    assert np.linalg.norm(x - xd) <= 1e-6 * np.linalg.norm(xd)
