"""Mesh topology, geometry and the switch function (Sections 2.2, 3.1, 4.2).

* Faces are identified by their sorted vertex tuples; face i of a simplex is the
  face opposite its local vertex i, with the remaining vertices in local order.
* Interior faces are ordered by (smaller element, larger element); boundary
  faces by (element, local face).  An interior face is integrated on the vertex
  order it has in its smaller-numbered element.
* Boundary faces missing from the caller's tagged list are Dirichlet.
* Switch (Section 2.2): S_K^K' = -S_K'^K.  R4 (the paper defines a consistent
  switch in Section 4.2 but gives no construction): S_K^K' = sign(n_KK' . w)
  with w = (1, sqrt 2, sqrt 3) truncated to d, n_KK' the unit normal pointing
  from K to K'; when |n . w| < 1e-12 the larger element index gets +1.  The
  natural switch of Section 2.2 (S_K^K' > 0 iff N(K) > N(K')) is available with
  the element index or a caller enumeration as N.
* The element with S < 0 on a face is its "q-side": it takes u-hat from its
  neighbour and carries the boundary gradient q^f (eq. edge_flux_interior).
* R6: h_avg = mean over Dirichlet faces f of d |K_f| / |f| (the height of K_f
  over f), C_D = gamma / h_avg (Section 2.2, after eq. cdg_fluxes).
"""
from __future__ import annotations

import math
import numpy as np


def face_normal(fv: np.ndarray, opp: np.ndarray):
    """Unit normal of the face with vertices fv, pointing away from opp, and
    the face measure."""
    d = fv.shape[1]
    if d == 2:
        t = fv[1] - fv[0]
        n = np.array([t[1], -t[0]])
        meas = float(np.linalg.norm(t))
    else:
        n = np.cross(fv[1] - fv[0], fv[2] - fv[0])
        meas = 0.5 * float(np.linalg.norm(n))
    n = n / np.linalg.norm(n)
    if np.dot(n, opp - fv[0]) > 0:
        n = -n
    return n, meas


class Topology:
    def __init__(self, mesh, switch_kind: int = 0, face_switch=None, enumeration=None):
        self.d = d = mesh.dim
        self.xyz = np.asarray(mesh.xyz, dtype=np.float64)
        self.elem = np.asarray(mesh.elem, dtype=np.int64)
        ne = self.ne = len(self.elem)
        self.vol = np.zeros(ne)
        for K in range(ne):
            s = self.xyz[self.elem[K]]
            self.vol[K] = abs(np.linalg.det(s[1:] - s[0])) / math.factorial(d)
        table: dict[tuple, list] = {}
        for K in range(ne):
            for l in range(d + 1):
                key = tuple(sorted(int(v) for j, v in enumerate(self.elem[K]) if j != l))
                table.setdefault(key, []).append((K, l))
        tags = {}
        for fv, t in zip(np.asarray(mesh.bface), np.asarray(mesh.btag)):
            tags[tuple(sorted(int(v) for v in fv))] = int(t)
        interior, boundary = [], []
        for key, owners in table.items():
            if len(owners) == 2:
                (Ka, la), (Kb, lb) = sorted(owners)
                interior.append((Ka, Kb, la, lb))
            elif len(owners) == 1:
                K, l = owners[0]
                boundary.append((K, l, tags.get(key, 0)))
            else:
                raise ValueError("non-manifold face")
        interior.sort()
        boundary.sort()
        self.interior = interior
        self.boundary = boundary
        self.nbrs = [[] for _ in range(ne)]
        for (Ka, Kb, _, _) in interior:
            self.nbrs[Ka].append(Kb)
            self.nbrs[Kb].append(Ka)
        # geometry of interior faces, from the smaller element's side
        self.if_verts, self.if_n, self.if_meas = [], [], []
        for (Ka, Kb, la, lb) in interior:
            fv, opp = self.local_face(Ka, la)
            n, m = face_normal(fv, opp)
            self.if_verts.append(fv); self.if_n.append(n); self.if_meas.append(m)
        self.bf_verts, self.bf_n, self.bf_meas = [], [], []
        for (K, l, t) in boundary:
            fv, opp = self.local_face(K, l)
            n, m = face_normal(fv, opp)
            self.bf_verts.append(fv); self.bf_n.append(n); self.bf_meas.append(m)
        # switch S1[f] = S_{Ka}^{Kb} for interior face f = (Ka, Kb)
        if face_switch is not None:
            S1 = np.where(np.asarray(face_switch) > 0, 1, -1)
        elif switch_kind == 1:
            N = np.arange(ne) if enumeration is None else np.asarray(enumeration)
            S1 = np.array([1 if N[Ka] > N[Kb] else -1 for (Ka, Kb, _, _) in interior])
        else:
            w = np.array([1.0, math.sqrt(2.0), math.sqrt(3.0)])[:d]
            S1 = []
            for f, (Ka, Kb, _, _) in enumerate(interior):
                s = float(np.dot(self.if_n[f], w))
                if abs(s) < 1e-12:
                    S1.append(1 if Ka > Kb else -1)
                else:
                    S1.append(1 if s > 0 else -1)
            S1 = np.array(S1)
        self.S1 = S1.astype(np.int64)
        # q-side (S < 0) and u-side of each interior face
        self.qside = np.array([Ka if s < 0 else Kb for (Ka, Kb, _, _), s in zip(interior, S1)], dtype=np.int64)
        self.uside = np.array([Kb if s < 0 else Ka for (Ka, Kb, _, _), s in zip(interior, S1)], dtype=np.int64)
        dir_h = [d * self.vol[K] / m for (K, l, t), m in zip(boundary, self.bf_meas) if t == 0]
        if not dir_h:
            raise ValueError("the Dirichlet boundary must have positive measure")
        self.h_avg = float(np.mean(dir_h))

    def local_face(self, K: int, l: int):
        idx = [j for j in range(self.d + 1) if j != l]
        s = self.xyz[self.elem[K]]
        return s[idx], s[l]

    def simplex(self, K: int) -> np.ndarray:
        return self.xyz[self.elem[K]]
