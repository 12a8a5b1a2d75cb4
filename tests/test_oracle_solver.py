"""Pins of the oracle's V-cycle (R14) and PCG (R15): the V(nu, nu) cycle is a
symmetric positive definite linear operator; a one-level cycle is the exact
solve; the cycle equals the textbook multigrid error propagation
E = S^nu2 (I - L B_{l+1} L^T A_l) S^nu1, S = I - omega D^-1 A_l, written with
dense matrices (B = (I - E) A^-1, B = A^-1 on the coarsest level), for V(1,1),
V(2,2) and the paper's V(0,3); the k-th PCG iterate is the A-norm-optimal
(Galerkin) solution on the k-dimensional preconditioned Krylov space; PCG agrees
with a dense direct solve of A_0 u = b."""
import numpy as np
import pytest

from oracle.cdg import Level0
from oracle.hierarchy import MGHierarchy
from oracle.solver import VCycle, pcg
from synthetic import jittered_square, kuhn_cube, sin_source


@pytest.fixture(scope="module")
def setup():
    L0 = Level0(jittered_square(6), 2)
    H = MGHierarchy(L0, max_levels=3)
    return L0, H


def test_vcycle_symmetric_positive(setup):
    L0, H = setup
    V = VCycle(H.A, H.L, L0.np_, 2, 2)
    n = H.A[0].shape[0]
    B = np.stack([V.apply(e) for e in np.eye(n)], axis=1)
    assert np.abs(B - B.T).max() <= 1e-11 * np.abs(B).max()
    assert np.linalg.eigvalsh((B + B.T) / 2).min() > 0


def _closed_form(H, npb, nu1, nu2, omega=2.0 / 3.0):
    """B_0 from the error propagation recursion, bottom level up."""
    B = np.linalg.inv(H.A[-1].toarray())
    for l in range(len(H.A) - 2, -1, -1):
        A = H.A[l].toarray()
        n = A.shape[0]
        D = np.zeros_like(A)
        for K in range(n // npb):
            sl = slice(K * npb, (K + 1) * npb)
            D[sl, sl] = A[sl, sl]
        S = np.eye(n) - omega * np.linalg.solve(D, A)
        L = H.L[l].toarray()
        E = np.linalg.matrix_power(S, nu2) @ (np.eye(n) - L @ B @ L.T @ A) @ np.linalg.matrix_power(S, nu1)
        B = (np.eye(n) - E) @ np.linalg.inv(A)
    return B


@pytest.mark.parametrize("nu1,nu2", [(1, 1), (2, 2), (0, 3)])
def test_vcycle_equals_error_propagation_formula(setup, nu1, nu2):
    L0, H = setup
    V = VCycle(H.A, H.L, L0.np_, nu1, nu2)
    n = H.A[0].shape[0]
    Bv = np.stack([V.apply(e) for e in np.eye(n)], axis=1)
    Bc = _closed_form(H, L0.np_, nu1, nu2)
    assert np.abs(Bv - Bc).max() <= 1e-9 * np.abs(Bc).max()


@pytest.mark.parametrize("flexible", [False, True])
def test_pcg_iterates_are_krylov_galerkin_solutions(setup, flexible):
    """With x0 = 0 the k-th PCG iterate minimises the A-norm error over
    span{Bb, (BA)Bb, ..., (BA)^(k-1) Bb}, B the (fixed, SPD) V-cycle operator;
    computed here by a dense Galerkin solve on an orthonormalised basis of that
    space.  The recurrence residual equals b - A x_k."""
    L0, H = setup
    V = VCycle(H.A, H.L, L0.np_, 1, 1)
    A = H.A[0].toarray()
    n = A.shape[0]
    B = np.stack([V.apply(e) for e in np.eye(n)], axis=1)
    b = L0.rhs(sin_source(L0.all_volume_points()))
    K = [B @ b]
    for k in range(1, 7):
        Q, _ = np.linalg.qr(np.stack(K, axis=1))
        xg = Q @ np.linalg.solve(Q.T @ A @ Q, Q.T @ b)
        x, hist, it = pcg(H.A[0], b, V.apply, tol=0.0, maxit=k, flexible=flexible)
        assert it == k
        e = x - xg
        assert np.sqrt(e @ A @ e) <= 1e-9 * np.sqrt(xg @ A @ xg), k
        assert abs(hist[-1] - np.linalg.norm(b - A @ x) / np.linalg.norm(b)) <= 1e-10, k
        K.append(B @ (A @ K[-1]))


def test_single_level_is_direct_solve(setup):
    L0, H = setup
    V = VCycle(H.A[:1], [], L0.np_)
    b = np.random.default_rng(0).standard_normal(H.A[0].shape[0])
    x = V.apply(b)
    assert np.linalg.norm(H.A[0] @ x - b) <= 1e-8 * np.linalg.norm(b)


@pytest.mark.parametrize("flexible", [False, True])
def test_pcg_matches_dense_solve(setup, flexible):
    L0, H = setup
    V = VCycle(H.A, H.L, L0.np_, 1, 1)
    b = L0.rhs(sin_source(L0.all_volume_points()))
    x, hist, it = pcg(H.A[0], b, V.apply, tol=1e-12, flexible=flexible)
    xd = np.linalg.solve(H.A[0].toarray(), b)
    assert np.linalg.norm(x - xd) <= 1e-10 * np.linalg.norm(xd)
    assert hist[-1] <= 1e-12 and len(hist) == it + 1
    assert hist[0] == 1.0


def test_pcg_3d_and_zero_rhs():
    L0 = Level0(kuhn_cube(2), 1)
    H = MGHierarchy(L0, max_levels=3)
    V = VCycle(H.A, H.L, L0.np_, 1, 1)
    b = L0.rhs(sin_source(L0.all_volume_points()))
    x, hist, it = pcg(H.A[0], b, V.apply, tol=1e-10)
    xd = np.linalg.solve(H.A[0].toarray(), b)
    assert np.linalg.norm(x - xd) <= 1e-9 * np.linalg.norm(xd)
    x0, h0, it0 = pcg(H.A[0], np.zeros_like(b), V.apply)
    assert it0 == 0 and not x0.any()
