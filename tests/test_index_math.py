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


def test_f64_to_f32_rz_bits():
    """f64_to_f32_rz (the mixed form's residual hand-over) cuts the mantissa
    of a double to 24 bits with integer operations: the same as truncating
    toward zero in single precision for normal values, 0 below the smallest
    normal single.  Emulated bit for bit."""
    import struct

    def emu(x):
        b = struct.unpack("<Q", struct.pack("<d", x))[0]
        hi, lo = b >> 32, b & 0xFFFFFFFF
        sign = hi & 0x80000000
        e = ((hi >> 20) & 0x7FF) - 1023 + 127
        mant = ((hi & 0xFFFFF) << 3) | (lo >> 29)
        bits = sign if e <= 0 else (sign | 0x7F800000) if e >= 255 else (sign | (e << 23) | mant)
        return struct.unpack("<f", struct.pack("<I", bits))[0]

    rng = np.random.default_rng(11)
    xs = np.concatenate([rng.standard_normal(20000) * 10.0 ** rng.integers(-30, 30, 20000), [0.0, -0.0, 1.0, -2.5]])
    for x in xs:
        y = emu(float(x))
        f = np.float32(x)  # round to nearest
        # truncation: |y| <= |x|, same sign, and within one single-precision ulp of x
        assert abs(y) <= abs(x) and (y == 0 or np.sign(y) == np.sign(x))
        assert abs(x - y) <= abs(x) * 2.0 ** -23
        assert abs(float(f) - y) <= abs(x) * 2.0 ** -23
    assert emu(1e-40) == 0.0 and emu(3.0) == 3.0
