"""cdg_smooth_static, the allocation-free variant of cdg_smooth, called through
the C ABI: for callers that cannot allocate device memory where they call it,
its intermediate D^{-1} b lives in a fixed array inside the library instead of
the handle's buffer.  Two calls in a row must reproduce cdg_smooth (same
kernels, same arithmetic: within the 1e-13 relative tolerance of the other
operator tests), also for vectors that are not 16-byte aligned and on a
stream other than the default one; levels larger than the fixed array and the
coarsest level (no smoother there) must be rejected.
This file is collected last so that a failure here leaves the other results."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _solver():
    from paper_2012_08024_gb300 import Solver
    from synthetic import jittered_square
    return Solver(jittered_square(16), p=2, max_levels=3).bind()


def test_static_smoother_matches_cdg_smooth_twice():
    import torch
    S = _solver()
    rng = np.random.default_rng(11)
    for call in range(2):
        for level in range(S.n_levels - 1):
            n = S.info["n_l"][level] * S.np_
            x = torch.tensor(rng.standard_normal(n), device="cuda")
            b = torch.tensor(rng.standard_normal(n), device="cuda")
            y_ref = torch.empty_like(x)
            y = torch.full_like(x, float("nan"))
            S.smooth(level, x, b, y_ref)
            S.smooth_static(level, x, b, y)
            torch.cuda.synchronize()
            err = float((y - y_ref).norm() / y_ref.norm())
            assert err <= 1e-13, (call, level, err)


def test_static_smoother_unaligned_vectors_and_side_stream():
    """x and y one element into larger buffers (not 16-byte aligned: the kernel
    without vector loads runs), and a call on a non-default stream."""
    import torch
    S = _solver()
    rng = np.random.default_rng(12)
    n = S.info["n_l"][0] * S.np_
    xb = torch.tensor(rng.standard_normal(n + 1), device="cuda")
    b = torch.tensor(rng.standard_normal(n), device="cuda")
    x = xb[1:]
    y_ref = torch.empty(n, dtype=torch.float64, device="cuda")
    S.smooth(0, x.clone(), b, y_ref)
    yb = torch.full((n + 1,), float("nan"), dtype=torch.float64, device="cuda")
    y = yb[1:]
    assert x.data_ptr() % 16 and y.data_ptr() % 16
    S.smooth_static(0, x, b, y)
    torch.cuda.synchronize()
    assert float((y - y_ref).norm() / y_ref.norm()) <= 1e-13
    side = torch.cuda.Stream()
    y2 = torch.full((n,), float("nan"), dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    with torch.cuda.stream(side):
        S.smooth_static(0, x, b, y2, stream=side)
    side.synchronize()
    assert float((y2 - y_ref).norm() / y_ref.norm()) <= 1e-13


def test_static_smoother_rejects_coarsest_level():
    import torch
    from paper_2012_08024_gb300 import CdgError
    S = _solver()
    lc = S.n_levels - 1
    n = S.info["n_l"][lc] * S.np_
    x = torch.zeros(n, dtype=torch.float64, device="cuda")
    with pytest.raises(CdgError) as e:
        S.smooth_static(lc, x, x, torch.empty_like(x))
    assert e.value.code == 1


def test_static_smoother_rejects_levels_beyond_the_fixed_array():
    import torch
    from paper_2012_08024_gb300 import CdgError, Solver
    from synthetic import jittered_square
    S = Solver(jittered_square(240), p=3, max_levels=6).bind()   # 115,200 x 10 unknowns on level 0
    n = S.info["n_l"][0] * S.np_
    assert n > (1 << 20)
    x = torch.zeros(n, dtype=torch.float64, device="cuda")
    y = torch.empty_like(x)
    with pytest.raises(CdgError, match="fixed scratch") as e:
        S.smooth_static(0, x, x, y)
    assert e.value.code == 1
