"""Greedy element agglomeration (Section 3.2, Algorithm 2) applied
recursively (Section 3.1, Algorithm 1).

State: P = unprocessed elements; N(e) = number of distinct unprocessed
neighbours of e (R8: neighbours share a face of positive measure; at coarse
levels, any fine face); c(v) = number of unprocessed elements that contain
vertex v (R8: the vertex set of an agglomerate is the union of its children's
fine vertices).

Each step pops e_min = argmin over P of (N(e), e) (ties to the lowest index;
the paper is silent).
* N(e_min) >= 2: v_max = argmax over the vertices of e_min of c(v);
  E = {e_min} + {e in P containing v_max}; E leaves P and becomes a new block
  (children in the order e_min, then ascending index).
* N(e_min) < 2: e_min joins the adjacent already-built block with the fewest
  children.  R10: with no adjacent block yet, fall back to the first branch if
  N(e_min) >= 1, else e_min forms a block by itself.
After every step N(e) is again the number of e's neighbours left in P.
R9 (the random tie-breaks of Section 3.2 made implementation independent):
among tied candidates (vertices for v_max, blocks for the smallest block) pick
the smallest splitmix64(seed ^ (level << 48) ^ (e_min << 20) ^ candidate),
then the smallest candidate index.  splitmix64 is Steele, Lea and Flood's
SplitMix64 finaliser (constants 0x9E3779B97F4A7C15, 0xBF58476D1CE4E5B9,
0x94D049BB133111EB; shifts 30, 27, 31).
"""
from __future__ import annotations

import heapq

MASK = (1 << 64) - 1


def splitmix64(x: int) -> int:
    z = (x + 0x9E3779B97F4A7C15) & MASK
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK
    return z ^ (z >> 31)


def tie_key(seed: int, level: int, e_min: int, cand: int) -> int:
    return splitmix64((seed ^ (level << 48) ^ (e_min << 20) ^ cand) & MASK)


def greedy_agglomerate(verts: list[list[int]], nbrs: list[list[int]], seed: int, level: int):
    """One application of Algorithm 2.  Returns the blocks (lists of element
    indices of this level) in creation order."""
    n = len(verts)
    inc: dict[int, list[int]] = {}
    for e, vs in enumerate(verts):
        for v in vs:
            inc.setdefault(v, []).append(e)
    in_P = [True] * n
    N = [len(set(nb)) for nb in nbrs]
    c = {v: len(es) for v, es in inc.items()}
    heap = [(N[e], e) for e in range(n)]
    heapq.heapify(heap)
    blocks: list[list[int]] = []
    block_of = [-1] * n

    def remove(e):
        in_P[e] = False
        for v in verts[e]:
            c[v] -= 1

    def pop_min():
        while heap:
            k, e = heapq.heappop(heap)
            if in_P[e] and k == N[e]:
                return e
        return -1

    def decrement_neighbours(removed):
        for e in removed:
            for e2 in set(nbrs[e]):
                if in_P[e2]:
                    N[e2] -= 1
                    heapq.heappush(heap, (N[e2], e2))

    while True:
        e_min = pop_min()
        if e_min < 0:
            break
        remove(e_min)
        star = N[e_min] >= 2
        if not star:
            adj = sorted({block_of[e2] for e2 in nbrs[e_min] if block_of[e2] >= 0})
            if adj:
                best = min(adj, key=lambda B: (len(blocks[B]), tie_key(seed, level, e_min, B), B))
                blocks[best].append(e_min)
                block_of[e_min] = best
                decrement_neighbours([e_min])
                continue
            if N[e_min] >= 1:
                star = True
            else:
                block_of[e_min] = len(blocks)
                blocks.append([e_min])
                continue
        # vertex-star branch
        v_max = min(verts[e_min], key=lambda v: (-c[v], tie_key(seed, level, e_min, v), v))
        others = sorted(e for e in inc[v_max] if in_P[e])
        for e in others:
            remove(e)
        E = [e_min] + others
        B = len(blocks)
        for e in E:
            block_of[e] = B
        blocks.append(E)
        decrement_neighbours(E)
    return blocks


class Hierarchy:
    """Algorithm 1: repeated agglomeration, stopped at max_levels levels
    (including level 0) or when a level has a single element."""

    def __init__(self, elem_verts: list[list[int]], nbrs0: list[list[int]], max_levels: int, seed: int):
        self.verts = [[sorted(set(v)) for v in elem_verts]]
        self.nbrs = [[sorted(set(nb)) for nb in nbrs0]]
        self.members = [[[e] for e in range(len(elem_verts))]]   # fine elements of each element
        self.parent = []
        self.blocks = []
        while len(self.verts) < max_levels and len(self.verts[-1]) > 1:
            l = len(self.verts) - 1
            blocks = greedy_agglomerate(self.verts[-1], self.nbrs[-1], seed, l)
            par = [-1] * len(self.verts[-1])
            for B, es in enumerate(blocks):
                for e in es:
                    par[e] = B
            self.parent.append(par)
            self.blocks.append(blocks)
            self.verts.append([sorted(set(v for e in es for v in self.verts[-1][e])) for es in blocks])
            self.members.append([[m for e in es for m in self.members[-1][e]] for es in blocks])
            nb = [set() for _ in blocks]
            for e, es in enumerate(self.nbrs[-1]):
                for e2 in es:
                    if par[e] != par[e2]:
                        nb[par[e]].add(par[e2])
            self.nbrs.append([sorted(s) for s in nb])

    @property
    def n_levels(self):
        return len(self.verts)

    def tree_order(self):
        """Final numbering: the coarsest level keeps its creation order; on
        every finer level elements are sorted by (final index of the parent,
        own index), so the children of every agglomerate are contiguous.
        Returns order[l] = list of level-l indices in final order."""
        L = self.n_levels
        order = [None] * L
        order[L - 1] = list(range(len(self.verts[L - 1])))
        for l in range(L - 2, -1, -1):
            pos = {e: i for i, e in enumerate(order[l + 1])}
            order[l] = sorted(range(len(self.verts[l])), key=lambda e: (pos[self.parent[l][e]], e))
        return order
