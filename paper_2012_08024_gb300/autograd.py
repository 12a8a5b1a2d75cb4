"""torch.autograd.Function over the GB300 solve: u = A_0(kappa)^{-1} b(f, kappa).

Forward solves with the hierarchy of the current kappa (host set-up again when
kappa changes, since the operators and their coarsening depend on it).  Backward
runs the adjoint solve A_0^T lambda = dL/du (A_0 symmetric: the same V-cycle
preconditioned CG) and the library's dL/df and dL/dkappa kernels.  Every step
runs in libcdgmg.so; this module only marshals tensors.
"""
from __future__ import annotations

import hashlib

import numpy as np
import torch

from . import Solver


class SolverCache:
    """One bound Solver per kappa (keyed by the bytes of kappa)."""

    def __init__(self, mesh, **opts):
        self.mesh = mesh
        self.opts = opts
        self.key = None
        self.solver = None

    def get(self, kappa: torch.Tensor, device) -> Solver:
        k = kappa.detach().double().cpu().numpy()
        key = hashlib.sha1(np.ascontiguousarray(k).tobytes()).hexdigest()
        if key != self.key:
            self.solver = None
            self.solver = Solver(self.mesh, kappa=k, **self.opts).bind(device)
            self.key = key
        return self.solver


class CDGSolve(torch.autograd.Function):
    """u = CDGSolve.apply(f_q, kappa, cache): f_q [n_elements][nq] (device,
    FP64), kappa [n_elements] (positive), cache a SolverCache for the mesh."""

    @staticmethod
    def forward(ctx, f_q, kappa, cache):
        S = cache.get(kappa, f_q.device)
        u, hist, it, rc = S.solve(f_q.contiguous())
        if rc != 0:
            raise RuntimeError(f"forward solve did not converge (code {rc}, {it} iterations)")
        ctx.solver = S
        ctx.save_for_backward(u)
        return u

    @staticmethod
    def backward(ctx, dLdu):
        (u,) = ctx.saved_tensors
        S = ctx.solver
        lam, hist, it, rc = S.solve_adjoint(dLdu.contiguous().double())
        if rc != 0:
            raise RuntimeError(f"adjoint solve did not converge (code {rc}, {it} iterations)")
        dLdf = S.rhs_adjoint(lam) if ctx.needs_input_grad[0] else None
        dLdk = S.kappa_gradient(lam, u) if ctx.needs_input_grad[1] else None
        return dLdf, dLdk, None
