"""The autotuner (block-row tiling of the block-sparse kernel; threads across
the right-hand sides, right-hand sides per thread and block rows per CTA of
the multi-right-hand-side kernel) changes
launch configurations only: every variant sums in the same order, so tuned and
untuned handles give bit-identical solves."""
import numpy as np
import pytest

from synthetic import jittered_square, sin_source, sine_combination_sources

pytestmark = pytest.mark.gpu


def _t(x):
    import torch
    return torch.as_tensor(np.ascontiguousarray(x), device="cuda")


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_tuned_solve_is_bit_identical(precision):
    from paper_2012_08024_gb300 import Solver
    mesh = jittered_square(40)
    kw = dict(p=3, max_levels=4, nu_pre=2, nu_post=2, precision=precision)
    St = Solver(mesh, autotune=True, **kw).bind()
    Su = Solver(mesh, autotune=False, **kw).bind()
    tun = St.tuning()
    assert tun[0]["apply64_unroll"] in (1, 2, 4) and tun[0]["residual64_unroll"] in (1, 2, 4)
    for l in range(St.n_levels - 1):
        assert tun[l]["vcycle_residual_unroll"] in (1, 2, 4)
        assert tun[l]["vcycle_smoother_unroll"] in (1, 2, 4)
    assert all(v == 2 for v in Su.tuning()[0].values())      # the untuned default
    xq, _, _ = St.quadrature_points()
    fq = _t(sin_source(xq))
    ut, ht, itt, rct = St.solve(fq)
    uu, hu, itu, rcu = Su.solve(fq)
    assert rct == rcu == 0 and itt == itu
    assert np.array_equal(ht, hu)
    assert np.array_equal(ut.cpu().numpy(), uu.cpu().numpy())


def test_tuned_multi_rhs_is_bit_identical():
    from paper_2012_08024_gb300 import Solver
    mesh = jittered_square(20)
    R = 40
    kw = dict(p=2, max_levels=3, nu_pre=1, nu_post=1, precision="fp32", nrhs=R)
    St = Solver(mesh, autotune=True, **kw).bind()
    Su = Solver(mesh, autotune=False, **kw).bind()
    xq, _, _ = St.quadrature_points()
    fq = _t(sine_combination_sources(xq, R, mmax=4, seed0=5))
    ut, ht, itt, rct = St.solve_multi(fq)
    uu, hu, itu, rcu = Su.solve_multi(fq)
    assert rct == rcu == 0 and np.array_equal(itt, itu)
    assert np.array_equal(ut.cpu().numpy(), uu.cpu().numpy())
    tun = St.tuning()
    assert tun[0]["multi_apply64_tile"] in (32, 64) and tun[0]["multi_apply64_rows"] in (1, 2, 4)
    # a tile of at most 64 columns (R = 40): one or two columns per thread
    assert tun[0]["multi_apply64_tile"] * tun[0]["multi_apply64_cols"] <= 64
    for l in range(St.n_levels - 1):
        t = tun[l]
        assert t["multi_smoother_tile"] in (32, 64) and t["multi_smoother_rows"] in (1, 2, 4)
        assert t["multi_residual_tile"] in (32, 64) and t["multi_residual_rows"] in (1, 2, 4)
        assert t["multi_smoother_tile"] * t["multi_smoother_cols"] <= 64
        assert t["multi_residual_tile"] * t["multi_residual_cols"] <= 64
    assert "multi_apply64_tile" not in Su.tuning()[0]


@pytest.mark.parametrize("precision", ["fp32", "bf16"])
def test_tuned_multi_rhs_256_columns_is_bit_identical(precision):
    """256 columns give the tuner tiles of up to 256 columns, two or four of
    them per thread; the tuned solve still equals the untuned one bit for bit."""
    from paper_2012_08024_gb300 import Solver
    mesh = jittered_square(24)
    R = 256
    kw = dict(p=3, max_levels=3, nu_pre=2, nu_post=2, precision=precision, nrhs=R, maxit=12)
    if precision == "bf16":
        kw["tensor_cores"] = False
    St = Solver(mesh, autotune=True, **kw).bind()
    Su = Solver(mesh, autotune=False, **kw).bind()
    xq, _, _ = St.quadrature_points()
    fq = _t(sine_combination_sources(xq, R, mmax=8, seed0=2))
    ut, ht, itt, rct = St.solve_multi(fq)
    uu, hu, itu, rcu = Su.solve_multi(fq)
    assert rct == rcu and np.array_equal(itt, itu)
    assert all(np.array_equal(a, b) for a, b in zip(ht, hu))
    assert np.array_equal(ut.cpu().numpy(), uu.cpu().numpy())
    tun = St.tuning()
    for l in range(St.n_levels - 1):
        assert tun[l]["multi_smoother_cols"] in (1, 2, 4) and tun[l]["multi_residual_cols"] in (1, 2, 4)
