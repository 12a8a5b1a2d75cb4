"""Pins of the oracle's V-cycle (R14) and PCG (R15): the V(nu, nu) cycle is a
symmetric positive definite linear operator; a one-level cycle is the exact
solve; PCG agrees with a dense direct solve of A_0 u = b."""
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
