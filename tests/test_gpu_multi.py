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


def test_tensor_core_smoother_matches_cuda_cores():
    """precision 2 smoother sweeps on tcgen05 (BF16 blocks exact in TF32, x
    split into two TF32 parts) against the same sweeps on CUDA cores: after
    one CG iteration the two differ by FP32 summation order only (amplified
    by the cancellation in x + omega (bh - x - Ahat x)), at least ten times
    less than the BF16 rounding of the blocks changes the iterate; R = 200
    spans a full and a ragged 128-column tile."""
    import torch
    from paper_2012_08024_gb300 import Solver
    mesh = jittered_square(10)
    R = 200
    out = {}
    for prec, tc in (("bf16", True), ("bf16", False), ("fp32", False)):
        S = Solver(mesh, p=3, max_levels=3, nu_pre=2, nu_post=2, precision=prec, nrhs=R, maxit=1,
                   tensor_cores=tc).bind()
        xq, _, _ = S.quadrature_points()
        fq = sine_combination_sources(xq, R, mmax=8, seed0=3)
        u, hists, its, rc = S.solve_multi(torch.tensor(fq, device="cuda"))
        out[prec, tc] = u.cpu().numpy()
    d_tc = rel(out["bf16", True], out["bf16", False])
    d_bf16 = rel(out["bf16", False], out["fp32", False])
    print(f"tensor cores vs CUDA cores {d_tc:.3g}, BF16 vs FP32 blocks {d_bf16:.3g}")
    assert d_tc <= 0.1 * d_bf16, (d_tc, d_bf16)


def test_tensor_core_multi_rhs_matches_oracle_p2():
    import torch
    from paper_2012_08024_gb300 import Solver
    mesh = jittered_square(14)
    R = 150
    S = Solver(mesh, p=2, max_levels=3, nu_pre=1, nu_post=1, precision="bf16", nrhs=R).bind()
    xq, _, _ = S.quadrature_points()
    fq = sine_combination_sources(xq, R, mmax=8, seed0=7)
    u, hists, its, rc = S.solve_multi(torch.tensor(fq, device="cuda"))
    assert rc == 0
    L0 = Level0(mesh, 2)
    A = L0.matrix().tocsc()
    lu = spl.splu(A)
    U = u.cpu().numpy()
    for r in range(0, R, 7):
        b = L0.rhs(fq[r])
        assert rel(U[r].ravel(), lu.solve(b)) <= 1e-9


def test_tensor_core_wait_timeout_is_reported_and_recoverable():
    """Failure detection without a fault: with the loop-wait limit of the tcgen05
    sweep set to 0 from the host, the first wait of the first sweep gives up at
    once; the kernel drains its issued MMAs (default limit), frees its tensor
    memory and flags the timeout, and cdg_solve_multi returns CDG_ETIMEOUT.
    With the limit restored, the same bound handle solves to the oracle's
    direct solutions."""
    import torch
    from paper_2012_08024_gb300 import CdgError, Solver
    mesh = jittered_square(14)
    R = 150
    S = Solver(mesh, p=2, max_levels=3, nu_pre=1, nu_post=1, precision="bf16", nrhs=R).bind()
    xq, _, _ = S.quadrature_points()
    fq = torch.tensor(sine_combination_sources(xq, R, mmax=8, seed0=7), device="cuda")
    S.set_wait_limit(0)
    with pytest.raises(CdgError) as e:
        S.solve_multi(fq)
    assert e.value.code == 6 and "iteration limit" in str(e.value)
    torch.cuda.synchronize()
    S.set_wait_limit(-1)
    u, hists, its, rc = S.solve_multi(fq)
    assert rc == 0
    L0 = Level0(mesh, 2)
    A = L0.matrix().tocsc()
    lu = spl.splu(A)
    U = u.cpu().numpy()
    for r in range(0, R, 7):
        assert rel(U[r].ravel(), lu.solve(L0.rhs(fq[r].cpu().numpy()))) <= 1e-9


def _exported_A0(S):
    import scipy.sparse as sp
    ex = S.export_level(0)
    npb = S.np_
    n = len(ex["rowptr"]) - 1
    return sp.bsr_matrix((ex["val"], ex["col"], ex["rowptr"]), shape=(n * npb, n * npb)).tocsr()


@pytest.mark.parametrize("p,R,m", [(3, 200, 12), (2, 96, 12), (3, 256, 40)])
def test_tc_fp64_apply_matches_fp64(p, R, m):
    """The FP64 level-0 apply by exact splitting on tcgen05 (tc_fp64_apply)
    against the library's own A_0 applied in FP64 by scipy, column by column,
    on columns whose scales spread over e^+-6 and a zero column, R spanning a
    full and a ragged 128-column tile: relative error <= 1e-13 per column (the
    split truncates below 2^-56 of the row and column scales).  On the 40 x 40
    mesh every CTA runs about ten block rows, so both TMEM accumulator sets
    and every stage of the copy ring are reused many times.  The FP64
    CUDA-core apply of the same handle type is held to 1e-14."""
    import torch
    from paper_2012_08024_gb300 import Solver
    mesh = jittered_square(m)
    rng = np.random.default_rng(41)
    for tc in (True, False):
        S = Solver(mesh, p=p, max_levels=3, precision="fp32", nrhs=R, tc_fp64_apply=tc).bind()
        A = _exported_A0(S)
        n = A.shape[0]
        X = rng.standard_normal((n, R)) * np.exp(rng.uniform(-6, 6, R))[None, :]
        X[:, 5] = 0.0
        x = torch.tensor(X, device="cuda")
        y = torch.empty_like(x)
        S.apply_multi(x, y)
        Y = y.cpu().numpy()
        ref = A @ X
        nr = np.linalg.norm(ref, axis=0)
        err = np.linalg.norm(Y - ref, axis=0) / np.where(nr > 0, nr, 1.0)
        assert not Y[:, 5].any()
        assert err.max() <= (1e-13 if tc else 1e-14), (tc, err.max())
        print(f"p={p} R={R} tensor-core split={tc}: worst column error {err.max():.2e}")


def test_tc_fp64_apply_solve_matches_oracle():
    """Many right-hand sides with the outer FP64 apply on tcgen05 (exact
    splitting): every column 1e-9 from the oracle's direct solution and true
    residual <= 2e-10 ||b|| by the oracle's operator."""
    import torch
    from paper_2012_08024_gb300 import Solver
    mesh = jittered_square(12)
    R = 140
    S = Solver(mesh, p=3, max_levels=3, nu_pre=2, nu_post=2, precision="fp32", nrhs=R, tc_fp64_apply=True).bind()
    xq, _, _ = S.quadrature_points()
    fq = sine_combination_sources(xq, R, mmax=8, seed0=11)
    u, hists, its, rc = S.solve_multi(torch.tensor(fq, device="cuda"))
    assert rc == 0
    L0 = Level0(mesh, 3)
    A = L0.matrix().tocsc()
    lu = spl.splu(A)
    U = u.cpu().numpy()
    for r in range(0, R, 9):
        b = L0.rhs(fq[r])
        assert hists[r][-1] <= 1e-10
        assert np.linalg.norm(b - A @ U[r].ravel()) <= 2e-10 * np.linalg.norm(b)
        assert rel(U[r].ravel(), lu.solve(b)) <= 1e-9


def test_tc_fp64_apply_wait_timeout_is_reported():
    """Failure detection without a fault in the split apply: with the loop-wait
    limit at 0 the first wait of each role (the issuing thread's wait for a
    stage's copies, the epilogue's wait for a finished row) gives up at once,
    the kernel drains its copies and MMAs and frees its tensor memory, and the
    call returns CDG_ETIMEOUT; with the limit restored the same handle applies
    within 1e-13."""
    import torch
    from paper_2012_08024_gb300 import CdgError, Solver
    S = Solver(jittered_square(10), p=3, max_levels=3, precision="fp32", nrhs=128, tc_fp64_apply=True).bind()
    A = _exported_A0(S)
    X = np.random.default_rng(3).standard_normal((A.shape[0], 128))
    x = torch.tensor(X, device="cuda")
    y = torch.empty_like(x)
    S.set_wait_limit(0)
    with pytest.raises(CdgError) as e:
        S.apply_multi(x, y)
    assert e.value.code == 6
    S.set_wait_limit(-1)
    S.apply_multi(x, y)
    ref = A @ X
    assert np.linalg.norm(y.cpu().numpy() - ref) <= 1e-13 * np.linalg.norm(ref)
