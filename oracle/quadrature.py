"""Quadrature on simplices (Section 3.3: agglomerate integrals are sums of
integrals over the sub-elements of the input mesh).

R3: collapsed-coordinate (Duffy) product rules built from Gauss-Legendre
points on [0, 1], exact for polynomials of total degree k:
  d=1: n = ceil((k+1)/2) points;
  d=2: xi1 = a(1-b), xi2 = b, weight w_a w_b (1-b),
       n_a = ceil((k+1)/2), n_b = ceil((k+2)/2);
  d=3: xi1 = a(1-b)(1-c), xi2 = b(1-c), xi3 = c, weight w_a w_b w_c (1-b)(1-c)^2,
       n_c = ceil((k+3)/2).
Points are enumerated with a outermost, then b, then c.
"""
from __future__ import annotations

import math
import numpy as np


def gauss_legendre_01(n: int):
    x, w = np.polynomial.legendre.leggauss(n)
    return 0.5 * (x + 1.0), 0.5 * w


def simplex_rule(d: int, k: int):
    """Reference points [nq][d] and weights [nq] on {xi >= 0, sum xi <= 1}."""
    if d == 1:
        t, w = gauss_legendre_01(math.ceil((k + 1) / 2))
        return t[:, None].copy(), w.copy()
    na = math.ceil((k + 1) / 2)
    nb = math.ceil((k + 2) / 2)
    a, wa = gauss_legendre_01(na)
    b, wb = gauss_legendre_01(nb)
    pts, wts = [], []
    if d == 2:
        for ia in range(na):
            for ib in range(nb):
                pts.append((a[ia] * (1 - b[ib]), b[ib]))
                wts.append(wa[ia] * wb[ib] * (1 - b[ib]))
        return np.array(pts), np.array(wts)
    nc = math.ceil((k + 3) / 2)
    c, wc = gauss_legendre_01(nc)
    for ia in range(na):
        for ib in range(nb):
            for ic in range(nc):
                pts.append((a[ia] * (1 - b[ib]) * (1 - c[ic]), b[ib] * (1 - c[ic]), c[ic]))
                wts.append(wa[ia] * wb[ib] * wc[ic] * (1 - b[ib]) * (1 - c[ic]) ** 2)
    return np.array(pts), np.array(wts)


def map_simplex(verts: np.ndarray, ref_pts: np.ndarray, ref_w: np.ndarray):
    """Physical points and weights on the simplex with vertices verts [m+1][d]
    (m = dimension of the simplex, d = ambient dimension)."""
    v0 = verts[0]
    E = verts[1:] - v0                      # [m][d]
    x = v0 + ref_pts @ E
    m = E.shape[0]
    if m == E.shape[1]:
        scale = abs(np.linalg.det(E))
    else:                                   # face of a d-simplex: m! * measure
        scale = math.sqrt(abs(np.linalg.det(E @ E.T)))
    return x, ref_w * scale
