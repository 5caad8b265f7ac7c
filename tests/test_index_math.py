"""Host check of the division-free index arithmetic the tail kernel uses
(small_div in chhs_kernels.cuh): for 0 <= t < 2^21 and d >= 1, truncating
(t + 1/2) * rn(1/d) in single precision gives t // d exactly.  IEEE single
precision is emulated with numpy float32 (round to nearest, no contraction:
the device expression is an add followed by a multiply)."""
import numpy as np
import pytest


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


def _quad_tile(nx):
    """quad_tile in chhs_corr3.cuh restated: (lq, ly, lz) of a block's brick."""
    nq = nx // 4
    lq = 0
    while (1 << lq) < nq and lq < 5:
        lq += 1
    rem = 7 - lq
    lz = rem >> 1
    return lq, rem - lz, lz


def _quad_pass_accesses(nx, ny, nz, block=128):
    """Every thread of a k_smooth_c4 launch on an nx x ny x nz level (nx a
    multiple of 4), with the kernel's index arithmetic restated: the grid of
    bricks (quad_grid), the quad each live thread takes."""
    lq, ly, lz = _quad_tile(nx)
    assert (1 << (lq + ly + lz)) == block
    nq = nx // 4
    gx, gy, gz = -(-nq // (1 << lq)), -(-ny // (1 << ly)), -(-nz // (1 << lz))
    bx, by, bz, tid = np.meshgrid(np.arange(gx), np.arange(gy), np.arange(gz), np.arange(block), indexing="ij")
    q = (bx << lq) + (tid & ((1 << lq) - 1))
    j = (by << ly) + ((tid >> lq) & ((1 << ly) - 1))
    k = (bz << lz) + (tid >> (lq + ly))
    live = (q < nq) & (j < ny) & (k < nz)
    return None, q[live].ravel(), j[live].ravel(), k[live].ravel()


@pytest.mark.parametrize("shape", [(128, 128, 128), (64, 64, 64), (32, 32, 32), (16, 16, 16), (8, 8, 8),
                                   (64, 32, 16), (16, 8, 24), (12, 6, 10), (4, 4, 4), (256, 256, 256),
                                   (20, 40, 8)])
def test_quad_pass_index_map(shape):
    """k_smooth_c4's thread-to-quad map and bounds: each quad of the level is
    taken by exactly one live thread of the grid of bricks (blocks of 128
    threads over 2^lq quads x 2^ly rows x 2^lz planes; the grid's y and z
    extents within the launch limit for these shapes), every 16-byte vector
    starts at a multiple of 4 cells and lies in
    the level, the outside x neighbour and the y/z neighbour quads are read
    only where they exist, and the coarse pairs of the prolongation lie in
    the coarser level and start at an even cell."""
    nx, ny, nz = shape
    assert nx % 4 == 0
    _, q, j, k = _quad_pass_accesses(nx, ny, nz)
    nq = nx // 4
    lq, ly, lz = _quad_tile(nx)
    assert -(-ny // (1 << ly)) <= 65535 and -(-nz // (1 << lz)) <= 65535
    assert np.array_equal(np.sort(q + nq * (j + ny * k)), np.arange(nq * ny * nz))
    assert q.min() >= 0 and q.max() < nq and j.min() >= 0 and j.max() < ny
    ncell = nx * ny * nz
    sy, sz = nx, nx * ny
    c4 = 4 * q + nx * (j + ny * k)
    assert (c4 % 4 == 0).all()
    ym, yp, zm, zp = j > 0, j + 1 < ny, k > 0, k + 1 < nz
    for colour in (0, 1):
        s = (j + k + colour) & 1
        xin = np.where(s == 1, 4 * q + 4 < nx, q > 0)
        xe = np.where(s == 1, c4 + 4, c4 - 1)
        loads = [c4] + [c4 + d for d, ok in ((-sy, ym), (sy, yp), (-sz, zm), (sz, zp))]
        oks = [np.ones_like(ym), ym, yp, zm, zp]
        for a, ok in zip(loads, oks):
            assert ((a[ok] >= 0) & (a[ok] + 3 < ncell)).all()
        assert ((xe[xin] >= 0) & (xe[xin] < ncell)).all()
        # the outside neighbour is the row's, and missing only at the row's ends
        assert (xe[xin] // nx == c4[xin] // nx).all()
        assert (~xin == np.where(s == 1, 4 * q + 4 == nx, q == 0)).all()
        # the updated cells 4q+s, 4q+s+2 are of the pass's colour
        for h in (0, 1):
            i = 4 * q + s + 2 * h
            assert ((i + j + k + colour) % 2 == 0).all() and (i < nx).all()
        if ny % 2 == 0 and nz % 2 == 0 and nx >= 4:
            cx, cy, cz = nx // 2, ny // 2, nz // 2
            cn = cx * cy * cz

            def crow(jj, kk):
                return cx * ((jj >> 1) + cy * (kk >> 1)) + 2 * q
            rows = [crow(j, k), crow(np.where(ym, j - 1, j), k), crow(np.where(yp, j + 1, j), k),
                    crow(j, np.where(zm, k - 1, k)), crow(j, np.where(zp, k + 1, k))]
            for a in rows:
                assert ((a >= 0) & (a + 1 < cn) & (a % 2 == 0)).all()
            ce = rows[0] + np.where(s == 1, 2, -1)
            assert ((ce[xin] >= 0) & (ce[xin] < cn)).all()
            assert (ce[xin] // cx == rows[0][xin] // cx).all()


def test_quad_pass_index_map_random_shapes():
    """The same checks on seeded random level shapes (x extents multiples of 4
    up to 512, y and z up to 96, even or odd)."""
    rng = np.random.default_rng(19)
    for _ in range(40):
        shape = (4 * int(rng.integers(1, 129)), int(rng.integers(1, 97)), int(rng.integers(1, 97)))
        test_quad_pass_index_map(shape)


def test_quad_component_selection():
    """The selections of k_smooth_c4's cell updates (at, xm, xp, put in
    smooth_c4_cells) restated: for the pass's two cells 4q+s+2h of a quad,
    `at` picks the cell's own component, xm and xp the components (or the
    outside neighbour e) at x - 1 and x + 1, and `put` writes the own one."""
    comps = "xyzw"

    def at(h, s):
        return ("w" if s else "z") if h else ("y" if s else "x")

    def xm(h, s):
        return ("z" if s else "y") if h else ("x" if s else "e")

    def xp(h, s):
        return ("e" if s else "w") if h else ("z" if s else "y")

    for s in (0, 1):
        e_off = 4 if s else -1  # the outside neighbour: 4q+4 when s = 1, 4q-1 when s = 0
        for h in (0, 1):
            own = s + 2 * h  # offset of the updated cell within the quad
            off = lambda c: e_off if c == "e" else comps.index(c)  # noqa: E731
            assert off(at(h, s)) == own
            assert off(xm(h, s)) == own - 1
            assert off(xp(h, s)) == own + 1
            # the missing-face rule: e falls back to the quad's end cell, which is
            # then the updated cell itself (4q when s = 0, 4q+3 when s = 1)
            if "e" in (xm(h, s), xp(h, s)):
                assert own == (3 if s else 0)
