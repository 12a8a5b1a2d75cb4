"""Shared helpers of the GPU parity tests: build the oracle objects and move
vectors between the oracle's working numbering and the library's tree order."""
import numpy as np

from oracle.cdg import Level0
from oracle.hierarchy import MGHierarchy
from oracle.solver import VCycle


class OracleCase:
    def __init__(self, mesh, p, max_levels, nu=1, seed=0, kappa=None, switch_kind=0):
        self.L0 = Level0(mesh, p, kappa=kappa, switch_kind=switch_kind)
        self.H = MGHierarchy(self.L0, max_levels=max_levels, seed=seed)
        self.order = self.H.agg.tree_order()
        self.npb = self.L0.np_
        self.V = VCycle(self.H.A, self.H.L, self.npb, nu, nu)

    def to_work(self, l, x_tree):
        x = np.asarray(x_tree).reshape(-1, self.npb)
        out = np.empty_like(x)
        out[self.order[l]] = x
        return out.ravel()

    def to_tree(self, l, x_work):
        x = np.asarray(x_work).reshape(-1, self.npb)
        return x[self.order[l]].ravel()


def rel(a, b):
    a, b = np.asarray(a).ravel(), np.asarray(b).ravel()
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)

