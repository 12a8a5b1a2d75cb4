"""cdg_smooth_static, the allocation-free variant of cdg_smooth, called through
the C ABI: for callers that cannot allocate device memory where they call it,
its intermediate D^{-1} b lives in a fixed array inside the library instead of
the handle's buffer.  Two calls in a row must reproduce cdg_smooth (same
kernels, same arithmetic: within the 1e-13 relative tolerance of the other
operator tests), and levels larger than the fixed array must be rejected.
This file is collected last so that a failure here leaves the other results."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_static_smoother_matches_cdg_smooth_twice():
    import torch
    from paper_2012_08024_gb300 import Solver
    from synthetic import jittered_square
    S = Solver(jittered_square(16), p=2, max_levels=3).bind()
    rng = np.random.default_rng(11)
    for call in range(2):
        for level in range(S.n_levels - 1):
            n = S.info["n_l"][level] * S.np_
            x = torch.tensor(rng.standard_normal(n), device="cuda")
            b = torch.tensor(rng.standard_normal(n), device="cuda")
            y_ref = torch.empty_like(x)
            y = torch.full_like(x, float("nan"))
            S.smooth(level, x, b, y_ref)
            rc = S.smooth_static(level, x, b, y)
            torch.cuda.synchronize()
            assert rc == 0
            err = float((y - y_ref).norm() / y_ref.norm())
            assert err <= 1e-13, (call, level, err)


def test_static_smoother_rejects_levels_beyond_the_fixed_array():
    import torch
    from paper_2012_08024_gb300 import CDG_MAX_LEVELS, Solver, lib
    from synthetic import jittered_square
    S = Solver(jittered_square(240), p=3, max_levels=6).bind()   # 115,200 x 10 unknowns on level 0
    n = S.info["n_l"][0] * S.np_
    assert n > (1 << 20)
    x = torch.zeros(n, dtype=torch.float64, device="cuda")
    y = torch.empty_like(x)
    rc = S.smooth_static(0, x, x, y)
    assert rc == 1 and "fixed scratch" in lib().cdg_last_error(S._h).decode()
