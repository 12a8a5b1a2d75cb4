"""Many right-hand sides on one mesh (cdg_solve_multi) against the oracle: the
V-cycle runs on FP32 or BF16 block copies, the outer CG is FP64, so every
column must reach the FP64 tolerance: true residual <= 2e-10 ||b_r|| by the
oracle's operator and relative L2 <= 1e-9 from the oracle's direct solution
(the column's own CG stops at ||r|| <= 1e-10 ||b||)."""
import numpy as np
import pytest
import scipy.sparse.linalg as spl

from oracle.cdg import Level0
from synthetic import jittered_square, sine_combination_sources
from tests.gpu_common import rel

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision", ["fp32", "bf16"])
def test_multi_rhs_matches_oracle(precision):
    import torch
    from paper_2012_08024_gb300 import Solver
    mesh = jittered_square(12)
    R = 12
    S = Solver(mesh, p=3, max_levels=3, nu_pre=2, nu_post=2, precision=precision, nrhs=R).bind()
    xq, _, _ = S.quadrature_points()
    fq = sine_combination_sources(xq, R, mmax=8, seed0=0)
    u, hists, its, rc = S.solve_multi(torch.tensor(fq, device="cuda"))
    assert rc == 0
    L0 = Level0(mesh, 3)
    A = L0.matrix().tocsc()
    lu = spl.splu(A)
    U = u.cpu().numpy()
    for r in range(R):
        b = L0.rhs(fq[r])
        ud = lu.solve(b)
        assert hists[r][-1] <= 1e-10
        assert np.linalg.norm(b - A @ U[r].ravel()) <= 2e-10 * np.linalg.norm(b)
        assert rel(U[r].ravel(), ud) <= 1e-9, (r, rel(U[r].ravel(), ud))
    print(f"{precision} multi-RHS iterations per column: {list(its)}")


def test_bf16_blocks_are_used():
    """The BF16 V-cycle differs from the FP32 one by BF16 rounding (~1e-3),
    far above FP32 rounding: the two precision modes really differ."""
    import torch
    from paper_2012_08024_gb300 import Solver
    mesh = jittered_square(8)
    out = {}
    for prec in ("fp32", "bf16"):
        S = Solver(mesh, p=2, max_levels=3, precision=prec, nrhs=4, maxit=1).bind()
        xq, _, _ = S.quadrature_points()
        fq = sine_combination_sources(xq, 4, mmax=8, seed0=1)
        u, hists, its, rc = S.solve_multi(torch.tensor(fq, device="cuda"))
        out[prec] = u.cpu().numpy()
    d = rel(out["bf16"], out["fp32"])
    assert 1e-5 < d < 1e-1, d
