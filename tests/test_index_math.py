"""Host check of the division-free index arithmetic the tail kernel uses
(small_div in chhs_kernels.cuh): for 0 <= t < 2^21 and d >= 1, truncating
(t + 1/2) * rn(1/d) in single precision gives t // d exactly.  IEEE single
precision is emulated with numpy float32 (round to nearest, no contraction:
the device expression is an add followed by a multiply)."""
import numpy as np


def small_div(t, d):
    rd = np.float32(1.0) / d.astype(np.float32)
    x = t.astype(np.float32) + np.float32(0.5)
    return np.trunc(x * rd).astype(np.int64)


def test_small_div_exhaustive_small_range():
    # every t < 4096 against every d <= 4096 (tail levels hold at most a few thousand cells)
    t = np.arange(4096, dtype=np.int64)
    for d0 in range(1, 4097, 256):
        d = np.arange(d0, min(d0 + 256, 4097), dtype=np.int64)
        T, D = np.meshgrid(t, d, indexing="ij")
        assert np.array_equal(small_div(T, D), T // D)


def test_small_div_sampled_full_range():
    rng = np.random.default_rng(7)
    t = rng.integers(0, 1 << 21, size=2_000_000, dtype=np.int64)
    d = rng.integers(1, 1 << 21, size=t.size, dtype=np.int64)
    assert np.array_equal(small_div(t, d), t // d)
    # quotients near integers: t = q d - 1, q d, q d + d - 1
    d = rng.integers(1, 2048, size=200_000, dtype=np.int64)
    q = rng.integers(0, (1 << 21) // 2048, size=d.size, dtype=np.int64)
    for t in (q * d, q * d + d - 1, np.maximum(q * d - 1, 0)):
        assert np.array_equal(small_div(t, d), t // d)


def test_count_value_bits():
    """count_value<double> assembles n (1 <= n < 2^20) from its bits:
    exponent floor(log2 n) and n shifted into the 20 high mantissa bits."""
    import struct
    for n in list(range(1, 4097)) + [(1 << 20) - 1]:
        e = n.bit_length() - 1  # 31 - clz(n)
        hi = ((1023 + e) << 20) | ((n << (20 - e)) & 0xFFFFF)
        assert struct.unpack("<d", struct.pack("<Q", hi << 32))[0] == float(n)
