"""chhs_autotune: the autotuner of launch shapes and coarse sweep counts leaves
the run's state exactly as it was, picks one of its candidates, and the tuned
handle's next steps still match the oracle within the form's tolerance."""
import numpy as np
import pytest

from paper_1611_02967_gb300 import chhs, inputs
from test_gpu_parity import PHI_TOL, _check_step

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("shape", [(128, 128), (16, 16, 16)])
def test_autotune_keeps_state_and_steps_match_oracle(shape, precision):
    h, eps, gamma, dt = 0.05, 0.05, 2.0, 0.01
    phi0 = inputs.spinodal(shape, 41, mean=0.0, amplitude=0.4)
    with chhs.Run(shape, h, eps, gamma, dt, opts=chhs.default_opts(precision=precision)) as run:
        run.set_phi(phi0)
        run.step(2)
        before = run.get_state()
        t = run.autotune(2)
        after = run.get_state()
        for a, b in zip(before, after):
            assert np.array_equal(a, b)
        assert t["ms_per_step"] > 0
        if precision == 0:
            assert t["tail_cells"] in (64, 256, 512) and t["split_threads"] in (0, 8192, 32768)
        elif len(shape) == 2:
            assert t["tail_cells"] in (256, 1024, 2048) and t["tile_threads"] in (256, 512)
            assert (t["tile_w"], t["tile_h"]) in ((32, 16), (32, 32), (64, 16))
            assert t["small_tile"] in ((t["tile_w"], t["tile_h"], t["tile_threads"]), (16, 8, 256))
        else:
            assert t["tail_cells"] in (64, 512)
        assert (t["coarse_nu1"], t["coarse_nu2"]) in ((2, 2), (1, 1))
        for _ in range(2):
            _check_step(run, h, eps, gamma, dt, PHI_TOL[precision])


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("shape", [(256, 256), (32, 32, 32)])
def test_one_coarse_sweep_reaches_the_same_answer(shape, precision):
    """The coarse sweep counts and tile shapes the autotuner may choose change
    only the path to the solution: with one sweep each way below the finest
    level and 64 x 16 or 32 x 32 tiles (chhs_set_tuning) the steps still
    equal the oracle's, and the state is kept across the rebuild."""
    h, eps, gamma, dt = (0.025, 0.05, 1.0, 0.005) if len(shape) == 2 else (0.05, 0.04, 2.0, 0.005)
    phi0 = inputs.spinodal(shape, 43, mean=0.0, amplitude=0.05)
    with chhs.Run(shape, h, eps, gamma, dt, opts=chhs.default_opts(precision=precision)) as run:
        run.set_phi(phi0)
        run.step(2)
        before = run.get_state()
        t = run.autotune(2)
        for tw, th in ((64, 16), (32, 32)):
            run.set_tuning(t["tail_cells"], t["split_threads"], t["tile_threads"], 1, 1, tw, th)
            for a, b in zip(before, run.get_state()):
                assert np.array_equal(a, b)
            _check_step(run, h, eps, gamma, dt, PHI_TOL[precision])
            run.set_state(*before)
        with pytest.raises(chhs.ChhsError):
            run.set_tuning(t["tail_cells"], t["split_threads"], 100, 1, 1)  # not a multiple of 32
        _check_step(run, h, eps, gamma, dt, PHI_TOL[precision])


def test_small_tile_shape_changes_no_result():
    """The tiles of the levels under 512 x 256 cells (chhs_tuning.small_tile_*;
    here every level of a 256^2 run) only change how the colour passes are
    cut into blocks: the same steps with 16 x 8 tiles on 256 threads, 32 x
    16 on 512 and 8 x 8 on 64 are equal bit for bit (2D mixed form)."""
    shape, h, eps, gamma, dt = (256, 256), 0.025, 0.05, 1.0, 0.005
    phi0 = inputs.spinodal(shape, 47, mean=0.0, amplitude=0.05)
    out = []
    for ct in ((16, 8, 256), (32, 16, 512), (8, 8, 64)):
        with chhs.Run(shape, h, eps, gamma, dt, opts=chhs.default_opts(precision=1)) as run:
            run.set_tuning(1024, 8192, 512, 1, 1, 32, 16, 3, small_tile=ct)
            run.set_phi(phi0)
            _, v, _ = run.step(3)
            out.append((v, run.get_state()))
    for v, st in out[1:]:
        assert v == out[0][0]
        for a, b in zip(st, out[0][1]):
            assert np.array_equal(a, b)
