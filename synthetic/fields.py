"""Seeded source and coefficient fields, evaluated at caller-given points.

The manufactured solution is u = prod_i sin(pi x_i), so that -Laplace(u) = f with
f = d pi^2 prod_i sin(pi x_i) and u = 0 on the boundary of the unit square/cube.
"""
from __future__ import annotations

import numpy as np


def sin_solution(x: np.ndarray) -> np.ndarray:
    return np.prod(np.sin(np.pi * x), axis=-1)


def sin_source(x: np.ndarray) -> np.ndarray:
    d = x.shape[-1]
    return d * np.pi ** 2 * np.prod(np.sin(np.pi * x), axis=-1)


def sine_combination_sources(x: np.ndarray, nrhs: int, mmax: int = 8, seed0: int = 0) -> np.ndarray:
    """f_k(x) = sum_{m,n<=mmax} c_kmn sin(m pi x) sin(n pi y), c ~ N(0,1) from seed k.

    x: [..., 2]; returns [nrhs, ...]."""
    out = np.empty((nrhs,) + x.shape[:-1])
    m = np.arange(1, mmax + 1)
    sx = np.sin(np.pi * x[..., 0, None] * m)   # [..., mmax]
    sy = np.sin(np.pi * x[..., 1, None] * m)
    for k in range(nrhs):
        c = np.random.default_rng(seed0 + k).standard_normal((mmax, mmax))
        out[k] = np.einsum("...m,mn,...n->...", sx, c, sy)
    return out


def smoothed_lognormal_kappa(neighbors: list[np.ndarray], seed: int = 2) -> np.ndarray:
    """kappa = exp(g): g ~ N(0,1) per element, averaged once with its face
    neighbours, then rescaled to unit standard deviation (zero mean)."""
    n = len(neighbors)
    g = np.random.default_rng(seed).standard_normal(n)
    s = np.array([(g[i] + g[nb].sum()) / (1 + len(nb)) for i, nb in enumerate(neighbors)])
    s = (s - s.mean()) / s.std()
    return np.exp(s)
