"""The seeded inputs follow the stated recipe: element counts, jitter bounds,
fixed boundary, positive orientation, total measure, batch size distribution,
deterministic seeds, and the kappa field's unit log-deviation."""
import math

import numpy as np
import pytest

from synthetic import (batched_squares, face_neighbors, jittered_square, kuhn_cube, sine_combination_sources,
                       smoothed_lognormal_kappa)


def _signed_measure(mesh):
    p = mesh.xyz[mesh.elem]
    return np.linalg.det(p[:, 1:, :] - p[:, :1, :]) / math.factorial(mesh.dim)


@pytest.mark.parametrize("gen,n,jit,count", [(jittered_square, 16, 0.2, lambda n: 2 * n * n),
                                             (kuhn_cube, 5, 0.1, lambda n: 6 * n ** 3)],
                         ids=["square", "cube"])
def test_mesh_recipe(gen, n, jit, count):
    m = gen(n, seed=3)
    grid = gen(n, seed=3, jitter=0.0)
    assert m.n_elements == count(n) and m.n_vertices == (n + 1) ** m.dim
    d = m.xyz - grid.xyz
    on_boundary = np.any((grid.xyz < 1e-12) | (grid.xyz > 1 - 1e-12), axis=1)
    assert not d[on_boundary].any()                          # boundary vertices stay put
    assert np.abs(d).max() <= jit / n and np.abs(d[~on_boundary]).max() > 0.5 * jit / n
    vol = _signed_measure(m)
    assert vol.min() > 0                                      # positively oriented (Kuhn split reoriented)
    assert abs(vol.sum() - 1.0) < 1e-12                       # tiles the unit square / cube
    assert np.array_equal(gen(n, seed=3).xyz, m.xyz)          # deterministic
    assert not np.array_equal(gen(n, seed=4).xyz, m.xyz)


def test_batch_sizes_log_uniform():
    ms = batched_squares(64, 500, 20000, seed=1)
    t = np.array([m.n_elements for m in ms])
    assert len(ms) == 64 and t.min() >= 450 and t.max() <= 20500
    # log-uniform: the log sizes spread over the whole range, about half below the log midpoint
    lt = np.log(t)
    assert lt.min() < np.log(1000) and lt.max() > np.log(10000)
    assert 20 <= int((lt < 0.5 * (np.log(500) + np.log(20000))).sum()) <= 44


def test_sources_and_kappa():
    x = np.random.default_rng(0).uniform(size=(50, 2))
    f = sine_combination_sources(x, 3, mmax=8, seed0=0)
    assert f.shape == (3, 50)
    assert np.array_equal(f[1], sine_combination_sources(x, 1, mmax=8, seed0=1)[0])   # column k uses seed k
    edge = np.stack([np.zeros(5), np.linspace(0, 1, 5)], axis=1)
    assert np.abs(sine_combination_sources(edge, 2)).max() < 1e-12                   # zero on x = 0
    m = kuhn_cube(3)
    k = smoothed_lognormal_kappa(face_neighbors(m), seed=2)
    g = np.log(k)
    assert k.shape == (m.n_elements,) and k.min() > 0
    assert abs(g.mean()) < 1e-12 and abs(g.std() - 1.0) < 1e-12
