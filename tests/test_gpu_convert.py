"""FP64 -> FP32 rounding of the library (integer-pipe path plus the conversion instruction at the
range edges) against torch's cast, bit for bit."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from paper_1912_09056_gb300 import amgc  # noqa: E402


def _bits_from(hi_lo):
    return np.asarray(hi_lo, dtype=np.uint64).view(np.float64)


def _cases():
    rng = np.random.default_rng(7)
    # values across the whole FP64 exponent range, both signs
    e = rng.integers(0, 2047, 200000, dtype=np.uint64)
    frac = rng.integers(0, 1 << 52, 200000, dtype=np.uint64)
    sign = rng.integers(0, 2, 200000, dtype=np.uint64)
    wide = _bits_from((sign << np.uint64(63)) | (e << np.uint64(52)) | frac)
    # FP32's normal range, with the 29 dropped bits exactly at, just below and just above half an
    # FP32 ulp (ties to even, both parities of the kept bit)
    e2 = rng.integers(897, 1151, 60000, dtype=np.uint64)
    keep = rng.integers(0, 1 << 23, 60000, dtype=np.uint64)
    drop = np.array([1 << 28, (1 << 28) - 1, (1 << 28) + 1, 0, (1 << 29) - 1], dtype=np.uint64)
    d = drop[rng.integers(0, drop.size, 60000)]
    ties = _bits_from((e2 << np.uint64(52)) | (keep << np.uint64(29)) | d)
    # edges: the largest FP32 and the rounding boundary to infinity, the smallest normal and the
    # subnormal range, zeros, infinities, NaN
    f32max = float(np.finfo(np.float32).max)
    edges = np.array([0.0, -0.0, np.inf, -np.inf, np.nan, f32max, -f32max,
                      np.nextafter(f32max, np.inf), 3.4028235677973366e38, 3.4028235677973362e38,
                      1.1754943508222875e-38, 1.1754942e-38, 1e-39, -1e-40, 1.4e-45, 7e-46, 1e-50,
                      1.0, -1.0, 0.1, 1.0 / 3.0, 2.0 ** 127, 2.0 ** 128, 2.0 ** -126, 2.0 ** -127])
    return np.concatenate([wide, ties, -ties, edges])


def test_f64_to_f32_matches_the_cast_bit_for_bit():
    x = torch.from_numpy(_cases()).cuda()
    y = torch.empty(x.numel(), dtype=torch.float32, device="cuda")
    amgc.f64_to_f32(x, y)
    ref = x.float()
    got, want = y.cpu().numpy(), ref.cpu().numpy()
    nan = np.isnan(want)
    assert np.array_equal(np.isnan(got), nan)
    assert np.array_equal(got[~nan].view(np.uint32), want[~nan].view(np.uint32))


def test_f64_to_f32_empty_and_invalid():
    x = torch.empty(0, dtype=torch.float64, device="cuda")
    y = torch.empty(0, dtype=torch.float32, device="cuda")
    amgc.f64_to_f32(x, y)
    lib = amgc.load()
    assert lib.amgc_f64_to_f32(-1, 0, 0, None) == amgc.AMGC_EINVAL
    assert lib.amgc_f64_to_f32(4, 0, 0, None) == amgc.AMGC_EINVAL
