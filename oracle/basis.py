"""Modal bases on elements and agglomerates (Section 3.3).

R2: on every element or agglomerate E take the monomials of total degree <= p
in (x - c_E)/h_E, graded by degree and, within a degree, in descending
lexicographic order of the exponent tuple; c_E is the volume-weighted centroid,
h_E = max |v - c_E| over the vertices of E.  The monomials are orthonormalised
in L2(E) through the Cholesky factor of their exact Gram matrix, Gram = R R^T,
phi = R^{-1} m, so that the mass matrix on every level is the identity.
"""
from __future__ import annotations

import itertools
import math
import numpy as np

from .quadrature import simplex_rule, map_simplex


def exponents(d: int, p: int) -> list[tuple[int, ...]]:
    out = []
    for t in range(p + 1):
        layer = [a for a in itertools.product(range(t + 1), repeat=d) if sum(a) == t]
        layer.sort(reverse=True)
        out.extend(layer)
    return out


def monomials(x: np.ndarray, c: np.ndarray, h: float, exps) -> np.ndarray:
    """Values [..., n_p] of the scaled monomials at points x [..., d]."""
    y = (x - c) / h
    cols = []
    for a in exps:
        v = np.ones(y.shape[:-1])
        for i, ai in enumerate(a):
            v = v * y[..., i] ** ai
        cols.append(v)
    return np.stack(cols, axis=-1)


def monomial_grads(x: np.ndarray, c: np.ndarray, h: float, exps) -> np.ndarray:
    """Gradients [..., n_p, d] of the scaled monomials."""
    y = (x - c) / h
    d = y.shape[-1]
    out = np.zeros(y.shape[:-1] + (len(exps), d))
    for j, a in enumerate(exps):
        for k in range(d):
            if a[k] == 0:
                continue
            v = np.full(y.shape[:-1], a[k] / h)
            for i, ai in enumerate(a):
                e = ai - 1 if i == k else ai
                v = v * y[..., i] ** e
            out[..., j, k] = v
    return out


class Basis:
    """Orthonormal P_p basis on a region given as a list of simplices."""

    def __init__(self, simplices: list[np.ndarray], p: int):
        self.p = p
        d = simplices[0].shape[1]
        self.d = d
        self.exps = exponents(d, p)
        vols, cents = [], []
        for s in simplices:
            vols.append(abs(np.linalg.det(s[1:] - s[0])) / math.factorial(d))
            cents.append(s.mean(axis=0))
        vols = np.array(vols)
        self.volume = vols.sum()
        self.c = (vols[:, None] * np.array(cents)).sum(axis=0) / self.volume
        allv = np.concatenate(simplices, axis=0)
        self.h = float(np.max(np.linalg.norm(allv - self.c, axis=1)))
        rp, rw = simplex_rule(d, 2 * p)
        gram = np.zeros((len(self.exps), len(self.exps)))
        for s in simplices:
            x, w = map_simplex(s, rp, rw)
            m = monomials(x, self.c, self.h, self.exps)
            gram += (m * w[:, None]).T @ m
        R = np.linalg.cholesky(gram)
        self.T = np.linalg.inv(R)           # phi = T m, T lower triangular

    def eval(self, x: np.ndarray) -> np.ndarray:
        return monomials(x, self.c, self.h, self.exps) @ self.T.T

    def grad(self, x: np.ndarray) -> np.ndarray:
        g = monomial_grads(x, self.c, self.h, self.exps)          # [..., n_p(m), d]
        return np.einsum("ij,...jk->...ik", self.T, g)            # [..., n_p, d]
