"""The 3D mixed form's colour passes on x-quads against the same passes on one
cell per thread.

With quad_passes = 1 (the default) a colour pass of a 3D single-precision
level whose x extent is a multiple of 4 gives each thread four consecutive
cells of a row, updates the two of the pass's colour and reads every field
as 16-byte vectors; with 0 every thread updates one cell.  Each cell's
arithmetic is the same in the same order -- missing boundary faces read the
cell's own value under a zero coefficient in both -- so the steps must
agree bit for bit: fields, V-cycle counts and final norms.  The cases reach
every kind of pass: plain sweeps, the first pre-smoothing sweep that
completes the FAS right-hand side on a coarse level, the first
post-smoothing sweep that adds the prolongation (to every value read on
colour 0, to the cell's own on colour 1), and the finest level's last pass
that adds the finished correction to the double-precision iterate (after a
plain pass with V(2,2), after the colour-1 prolongation pass with V(1,1));
with nu1 = 0 the coarse right-hand side runs as its own kernel.  Each case
runs with the one-block tail from 1024 cells (the default) and from 64, so
that small levels (8^3: two quads per row) run as colour passes too, and the
grid with an x extent of 20 runs its 10-cell level on one cell per thread
beside the quad level above it; the 256 x 8 x 8 grid runs long rows (whole
warps in one row) on its finest level and, with the right-hand side
completed, on its 128 x 4 x 4 level.
"""
import numpy as np
import pytest

from paper_1611_02967_gb300 import chhs, inputs

pytestmark = pytest.mark.gpu

# numpy shapes (nz, ny, nx), h, eps, gamma, dt
CASES = [
    ((32, 32, 32), 0.2, 0.08, 2.0, 0.005),
    ((16, 32, 64), 0.1, 0.05, 4.0, 0.005),   # non-cubic
    ((24, 8, 16), 0.1, 0.08, 0.0, 0.005),    # gamma = 0: the pressure decouples
    ((8, 40, 20), 0.1, 0.08, 1.0, 0.01),     # x extent 20, then 10 (one cell per thread)
    ((10, 6, 12), 0.2, 0.1, 2.0, 0.01),      # ragged coarsening (6 x 3 x 5 below)
    ((8, 8, 256), 0.1, 0.08, 2.0, 0.005),    # x extents 256 and 128
]


def _tuned(shape, h, eps, gamma, dt, nu, tail, quad):
    opts = chhs.default_opts(precision=1, nu1=nu[0], nu2=nu[1])
    run = chhs.Run(shape, h, eps, gamma, dt, opts=opts)
    # the mixed form's default launch settings but the tail size, with the pass layout chosen
    run.set_tuning(tail, 8192, 512, nu[0], nu[1], quad_passes=quad)
    return run


@pytest.mark.parametrize("tail", [1024, 64])
@pytest.mark.parametrize("nu", [(2, 2), (1, 1), (0, 2)])
@pytest.mark.parametrize("shape,h,eps,gamma,dt", CASES)
def test_quad_passes_bit_identical_to_one_cell_per_thread(shape, h, eps, gamma, dt, nu, tail):
    phi0 = inputs.spinodal(shape, 303, mean=-0.1, amplitude=0.5)
    out = []
    for quad in (1, 0):
        with _tuned(shape, h, eps, gamma, dt, nu, tail, quad) as run:
            run.set_phi(phi0)
            steps = [run.step(1) for _ in range(3)]
            out.append((steps, run.get_state()))
    (sa, xa), (sb, xb) = out
    assert [s[1] for s in sa] == [s[1] for s in sb]  # V-cycles per step
    assert [s[2] for s in sa] == [s[2] for s in sb]  # final norms, bit for bit
    for a, b in zip(xa, xb):
        assert np.array_equal(a, b)


def test_quad_passes_setting_checked():
    shape = (8, 8, 8)
    with chhs.Run(shape, 0.2, 0.1, 1.0, 0.01, opts=chhs.default_opts(precision=1)) as run:
        with pytest.raises(chhs.ChhsError):
            run.set_tuning(1024, 8192, 512, 2, 2, quad_passes=2)
        run.set_tuning(1024, 8192, 512, 2, 2, quad_passes=0)
        run.set_phi(inputs.spinodal(shape, 5, mean=0.0, amplitude=0.3))
        run.step(2)
