"""Seeded simplicial meshes shaped like the Poisson workloads of Section 5.

The paper's own meshes (uniform n x n squares, a NACA-airfoil channel) are not
available; these generators stand in for them:

* ``jittered_square(n)``: the unit square cut into n x n cells, each split into
  two triangles along the (i, j) -> (i+1, j+1) diagonal; interior vertices are
  moved by U(-0.2h, 0.2h) per coordinate (numpy ``default_rng(seed)``, one draw
  of shape ((n+1)^2, 2) in row-major vertex order, boundary rows discarded).
* ``kuhn_cube(n)``: the unit cube cut into n^3 cells, each split into the six
  Kuhn tetrahedra around the (0,0,0) -> (1,1,1) diagonal, interior vertices
  moved by U(-0.1h, 0.1h) per coordinate (same draw rule); every tetrahedron is
  stored with positive orientation.  The 3D default jitter is half the 2D one:
  at 0.2h the Kuhn split produces sliver tetrahedra (dihedral angles near 163
  degrees) on which the CDG operator without interior penalty is indefinite.
* ``batched_squares``: many jittered squares with log-uniform triangle counts.
* ``square_with_holes``: a multiply connected domain (square with square holes).

Boundary faces are listed with a tag per face: 0 = Dirichlet, 1 = Neumann.
"""
from __future__ import annotations

from dataclasses import dataclass
import itertools
import numpy as np


@dataclass
class Mesh:
    dim: int
    xyz: np.ndarray     # [n_vertices][dim] float64
    elem: np.ndarray    # [n_elements][dim+1] int64
    bface: np.ndarray   # [n_bfaces][dim] int64
    btag: np.ndarray    # [n_bfaces] int32

    @property
    def n_elements(self) -> int:
        return int(self.elem.shape[0])

    @property
    def n_vertices(self) -> int:
        return int(self.xyz.shape[0])


def _boundary_faces(elem: np.ndarray, dim: int) -> np.ndarray:
    """Faces that belong to exactly one simplex (pure combinatorics)."""
    faces = []
    for i in range(dim + 1):
        cols = [c for c in range(dim + 1) if c != i]
        faces.append(elem[:, cols])
    f = np.concatenate(faces, axis=0)
    fs = np.sort(f, axis=1)
    uniq, inv, cnt = np.unique(fs, axis=0, return_inverse=True, return_counts=True)
    once = cnt[inv.ravel()] == 1
    return f[once]


def _tags(xyz: np.ndarray, bface: np.ndarray, neumann_axes: tuple[int, ...]) -> np.ndarray:
    """Tag 1 (Neumann) on faces lying on x_a = 0 or 1 for a in neumann_axes."""
    tags = np.zeros(len(bface), dtype=np.int32)
    for a in neumann_axes:
        c = xyz[bface][:, :, a]
        on = np.all(np.abs(c - 0.0) < 1e-12, axis=1) | np.all(np.abs(c - 1.0) < 1e-12, axis=1)
        tags[on] = 1
    return tags


def jittered_square(n: int, seed: int = 0, jitter: float = 0.2,
                    neumann_axes: tuple[int, ...] = ()) -> Mesh:
    h = 1.0 / n
    j, i = np.meshgrid(np.arange(n + 1), np.arange(n + 1), indexing="ij")
    xyz = np.stack([i.ravel() * h, j.ravel() * h], axis=1).astype(np.float64)
    rng = np.random.default_rng(seed)
    d = rng.uniform(-jitter * h, jitter * h, size=((n + 1) ** 2, 2))
    interior = ((i.ravel() > 0) & (i.ravel() < n) & (j.ravel() > 0) & (j.ravel() < n))
    xyz[interior] += d[interior]
    vid = lambda ii, jj: jj * (n + 1) + ii
    cj, ci = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    ci = ci.ravel(); cj = cj.ravel()
    v00 = vid(ci, cj); v10 = vid(ci + 1, cj); v11 = vid(ci + 1, cj + 1); v01 = vid(ci, cj + 1)
    t0 = np.stack([v00, v10, v11], axis=1)
    t1 = np.stack([v00, v11, v01], axis=1)
    elem = np.stack([t0, t1], axis=1).reshape(-1, 3).astype(np.int64)
    bface = _boundary_faces(elem, 2).astype(np.int64)
    return Mesh(2, xyz, elem, bface, _tags(xyz, bface, neumann_axes))


def kuhn_cube(n: int, seed: int = 0, jitter: float = 0.1,
              neumann_axes: tuple[int, ...] = ()) -> Mesh:
    h = 1.0 / n
    k, j, i = np.meshgrid(np.arange(n + 1), np.arange(n + 1), np.arange(n + 1), indexing="ij")
    xyz = np.stack([i.ravel() * h, j.ravel() * h, k.ravel() * h], axis=1).astype(np.float64)
    rng = np.random.default_rng(seed)
    d = rng.uniform(-jitter * h, jitter * h, size=((n + 1) ** 3, 3))
    ir, jr, kr = i.ravel(), j.ravel(), k.ravel()
    interior = ((ir > 0) & (ir < n) & (jr > 0) & (jr < n) & (kr > 0) & (kr < n))
    xyz[interior] += d[interior]
    vid = lambda a, b, c: (c * (n + 1) + b) * (n + 1) + a
    ck, cj, ci = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    ci, cj, ck = ci.ravel(), cj.ravel(), ck.ravel()
    tets = []
    for perm in itertools.permutations(range(3)):
        off = np.zeros(3, dtype=np.int64)
        vs = [vid(ci, cj, ck)]
        for ax in perm:
            off[ax] += 1
            vs.append(vid(ci + off[0], cj + off[1], ck + off[2]))
        tets.append(np.stack(vs, axis=1))
    elem = np.stack(tets, axis=1).reshape(-1, 4).astype(np.int64)
    p = xyz[elem]
    det = np.linalg.det(p[:, 1:, :] - p[:, :1, :])
    neg = det < 0
    elem[neg, 1], elem[neg, 2] = elem[neg, 2].copy(), elem[neg, 1].copy()
    bface = _boundary_faces(elem, 3).astype(np.int64)
    return Mesh(3, xyz, elem, bface, _tags(xyz, bface, neumann_axes))


def batched_squares(count: int = 64, tmin: int = 500, tmax: int = 20000, seed: int = 1) -> list[Mesh]:
    """Jittered squares with triangle counts log-uniform in [tmin, tmax]."""
    rng = np.random.default_rng(seed)
    t = np.exp(rng.uniform(np.log(tmin), np.log(tmax), size=count))
    ns = np.maximum(2, np.round(np.sqrt(t / 2.0)).astype(int))
    return [jittered_square(int(nn), seed=seed * 1000 + k) for k, nn in enumerate(ns)]


def square_with_holes(n: int, holes: tuple[tuple[int, int, int], ...] = ((2, 2, 1),),
                      seed: int = 0, jitter: float = 0.2) -> Mesh:
    """Jittered n x n square with square holes; hole = (i0, j0, size) in cells,
    counted on an n x n lattice.  All boundary faces (outer and hole) are Dirichlet."""
    m = jittered_square(n, seed=seed, jitter=0.0)
    keep = np.ones(m.n_elements, dtype=bool)
    for (i0, j0, s) in holes:
        for jj in range(j0, j0 + s):
            for ii in range(i0, i0 + s):
                c = jj * n + ii
                keep[2 * c] = False
                keep[2 * c + 1] = False
    elem = m.elem[keep]
    used = np.unique(elem)
    remap = -np.ones(m.n_vertices, dtype=np.int64)
    remap[used] = np.arange(len(used))
    xyz = m.xyz[used].copy()
    elem = remap[elem]
    bface = _boundary_faces(elem, 2).astype(np.int64)
    onb = np.zeros(len(xyz), dtype=bool)
    onb[np.unique(bface)] = True
    rng = np.random.default_rng(seed)
    h = 1.0 / n
    d = rng.uniform(-jitter * h, jitter * h, size=xyz.shape)
    xyz[~onb] += d[~onb]
    return Mesh(2, xyz, elem, bface, np.zeros(len(bface), dtype=np.int32))


def face_neighbors(mesh: Mesh) -> list[np.ndarray]:
    """Elements sharing a face with each element (combinatorics only)."""
    d = mesh.dim
    keys = {}
    for K, e in enumerate(mesh.elem):
        for i in range(d + 1):
            keys.setdefault(tuple(sorted(int(v) for j, v in enumerate(e) if j != i)), []).append(K)
    nb = [[] for _ in range(mesh.n_elements)]
    for owners in keys.values():
        if len(owners) == 2:
            a, b = owners
            nb[a].append(b)
            nb[b].append(a)
    return [np.array(sorted(x), dtype=np.int64) for x in nb]
