"""Pins of the oracle's quadrature (R3) and bases (R2, Section 3.3) against
closed forms: int over the reference simplex of xi^alpha = alpha! / (|alpha| + d)!
(Dirichlet integral), and Gram = I for the orthonormalised bases."""
import itertools
import math

import numpy as np
import pytest

from oracle.basis import Basis, exponents, monomials
from oracle.quadrature import simplex_rule, map_simplex
from synthetic import jittered_square, kuhn_cube


def exact_moment(alpha):
    d = len(alpha)
    return math.prod(math.factorial(a) for a in alpha) / math.factorial(sum(alpha) + d)


@pytest.mark.parametrize("d", [1, 2, 3])
@pytest.mark.parametrize("k", [0, 1, 2, 3, 4, 5, 6, 8])
def test_simplex_rule_exact_to_degree(d, k):
    x, w = simplex_rule(d, k)
    assert np.all(w > 0)
    for alpha in itertools.product(range(k + 1), repeat=d):
        if sum(alpha) > k:
            continue
        q = np.sum(w * np.prod(x ** np.array(alpha), axis=1))
        assert abs(q - exact_moment(alpha)) <= 1e-15 * max(1.0, exact_moment(alpha)) + 1e-16


def test_simplex_rule_point_counts():
    # n_a = ceil((k+1)/2), n_b = ceil((k+2)/2), n_c = ceil((k+3)/2)
    assert len(simplex_rule(2, 4)[1]) == 3 * 3
    assert len(simplex_rule(2, 6)[1]) == 4 * 4
    assert len(simplex_rule(3, 4)[1]) == 3 * 3 * 4
    assert len(simplex_rule(1, 6)[1]) == 4


def test_mapped_rule_measures():
    tri = np.array([[0.1, 0.2], [1.3, 0.4], [0.5, 1.7]])
    x, w = map_simplex(tri, *simplex_rule(2, 2))
    area = 0.5 * abs(np.linalg.det(tri[1:] - tri[0]))
    assert abs(w.sum() - area) < 1e-15
    # centroid is the mean of the vertices
    assert np.allclose((w[:, None] * x).sum(0) / area, tri.mean(0), atol=1e-15)
    face = np.array([[0.0, 0.0, 0.0], [2.0, 0.0, 0.0], [0.0, 3.0, 0.0]])
    x, w = map_simplex(face, *simplex_rule(2, 3))
    assert abs(w.sum() - 3.0) < 1e-14


def test_exponent_order():
    assert exponents(2, 2) == [(0, 0), (1, 0), (0, 1), (2, 0), (1, 1), (0, 2)]
    assert len(exponents(2, 3)) == 10 and len(exponents(3, 2)) == 10


@pytest.mark.parametrize("p", [1, 2, 3])
def test_basis_orthonormal_on_element_and_agglomerate(p):
    m = jittered_square(3)
    simp = [m.xyz[e] for e in m.elem]
    rp, rw = simplex_rule(2, 2 * p)
    for region in ([simp[4]], simp[2:9]):
        B = Basis(region, p)
        G = np.zeros((len(B.exps),) * 2)
        for s in region:
            x, w = map_simplex(s, rp, rw)
            ph = B.eval(x)
            G += (ph * w[:, None]).T @ ph
        assert np.abs(G - np.eye(len(B.exps))).max() < 1e-13
        # the orthonormal basis spans the monomials: T is invertible lower triangular
        assert np.allclose(np.triu(B.T, 1), 0.0)


def test_basis_gradient_matches_finite_difference():
    m = kuhn_cube(1)
    B = Basis([m.xyz[m.elem[2]]], 2)
    x = m.xyz[m.elem[2]].mean(0)
    g = B.grad(x[None])[0]
    h = 1e-6
    for k in range(3):
        e = np.zeros(3); e[k] = h
        fd = (B.eval((x + e)[None])[0] - B.eval((x - e)[None])[0]) / (2 * h)
        assert np.allclose(fd, g[:, k], atol=1e-7 * max(1, np.abs(g).max()))
