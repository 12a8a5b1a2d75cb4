"""The FP64 <-> FP32 conversion kernels (cdg_convert), which build their
results from the IEEE 754 bit fields with integer operations: bit for bit the
IEEE conversions (round to nearest, ties to even, for binary64 -> binary32;
exact for binary32 -> binary64), taken here from PyTorch's own CUDA casts, on
random bit patterns over the whole range and on the edge cases: exact ties
with even and odd kept parts, carries into the exponent and into infinity,
the boundaries of the normal binary32 range, subnormals, signed zeros,
infinities and NaN."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _doubles():
    rng = np.random.default_rng(5)
    bits = rng.integers(0, 2**63, size=200000, dtype=np.uint64) | (
        rng.integers(0, 2, size=200000, dtype=np.uint64) << np.uint64(63))
    wide = bits.view(np.float64)
    # exponents around the binary32 range, with random significands
    mid = rng.standard_normal(200000) * np.exp2(rng.integers(-160, 140, 200000))
    f = rng.standard_normal(5000).astype(np.float32).astype(np.float64)
    ulp = np.spacing(f.astype(np.float32)).astype(np.float64)
    ties = np.concatenate([f + ulp / 2, f - ulp / 2, f + ulp / 2 * (1 + 2**-30), f + ulp / 2 * (1 - 2**-30)])
    fmax = float(np.finfo(np.float32).max)
    tiny = float(np.finfo(np.float32).tiny)
    edge = np.array([0.0, -0.0, np.inf, -np.inf, np.nan, fmax, -fmax, fmax * (1 + 2**-25), fmax * (1 + 2**-24),
                     fmax * (1 + 2**-23), tiny, -tiny, tiny * (1 - 2**-30), tiny / 2, tiny * 2**-23, tiny * 2**-24,
                     tiny * 2**-25, 1.0 + 2**-24, 1.0 + 3 * 2**-24, 1.0 - 2**-25, 2.0 - 2**-24, 5e-324, 1e308])
    return np.concatenate([wide, mid, ties, edge])


def test_f64_to_f32_is_ieee_round_to_nearest_even():
    import torch
    from paper_2012_08024_gb300 import convert
    x = torch.tensor(_doubles(), device="cuda")
    got = convert(x)
    want = x.to(torch.float32)
    assert got.dtype == torch.float32
    g, w = got.cpu().numpy(), want.cpu().numpy()
    nan = np.isnan(w)
    assert np.array_equal(np.isnan(g), nan)
    assert np.array_equal(g[~nan].view(np.uint32), w[~nan].view(np.uint32))


def test_f32_to_f64_is_exact():
    import torch
    from paper_2012_08024_gb300 import convert
    rng = np.random.default_rng(6)
    bits = rng.integers(0, 2**32, size=400000, dtype=np.uint64).astype(np.uint32)
    edge = np.array([0.0, -0.0, np.inf, -np.inf, np.nan, 1e-45, -1e-45, 1.1754942e-38, 1.17549435e-38,
                     3.4028235e38], dtype=np.float32)
    f = np.concatenate([bits.view(np.float32), edge])
    x = torch.tensor(f, device="cuda")
    got = convert(x)
    want = x.to(torch.float64)
    assert got.dtype == torch.float64
    g, w = got.cpu().numpy(), want.cpu().numpy()
    nan = np.isnan(w)
    assert np.array_equal(np.isnan(g), nan)
    assert np.array_equal(g[~nan].view(np.uint64), w[~nan].view(np.uint64))


def test_convert_empty_and_errors():
    import torch
    from paper_2012_08024_gb300 import CdgError, convert, lib
    assert convert(torch.empty(0, dtype=torch.float64, device="cuda")).numel() == 0
    assert lib().cdg_convert(None, None, -1, 1, None) != 0
    assert lib().cdg_convert(None, None, 5, 1, None) != 0
    with pytest.raises(ValueError):
        convert(torch.zeros(3))
