"""The batched step (chhs_batch_*): many runs of uneven size in one graph of
batched launches, one launch per multigrid level over all runs.

Each run of a batch executes the same kernels on the same data with the same
block shapes as its own handle, so its results must be bit-identical to a
solo run (chhs_create with the same options), V-cycle counts included; and a
sampled run's step must match the oracle within the mixed-precision bound.
"""
import numpy as np
import pytest

import oracle
from paper_1611_02967_gb300 import chhs, inputs

pytestmark = pytest.mark.gpu

MIXED_TOL = 1e-8

RUNS_2D = [((64, 64), 0.025, 0.05, 1.0, 0.005),
           ((128, 128), 0.025, 0.03, 2.5, 0.005),
           ((256, 256), 0.025, 0.08, 0.5, 0.005),
           ((32, 96), 0.05, 0.05, 4.0, 0.005),      # non-square
           ((24, 40), 0.1, 0.08, 0.0, 0.01),        # ragged: a single level of 3 x 5 below 24 x 40, gamma 0
           ((2, 2), 0.5, 0.2, 1.0, 0.01)]           # the coarsest grid only: the tail is the whole V-cycle
RUNS_3D = [((16, 16, 16), 0.1, 0.08, 2.0, 0.005),
           ((32, 32, 32), 0.05, 0.04, 4.0, 0.005),
           ((16, 8, 12), 0.1, 0.08, 0.0, 0.005)]


def _phi0(shape, q):
    return inputs.spinodal(shape, 500 + q, mean=-0.05, amplitude=0.3)


@pytest.mark.parametrize("max_inner", [4, 2, 1])
@pytest.mark.parametrize("runs", [RUNS_2D, RUNS_3D], ids=["2d", "3d"])
def test_batch_bit_identical_to_solo_runs(runs, max_inner):
    """Each run takes the V-cycles its own norms ask for (up to max_inner
    between two norms), as it would alone."""
    nsteps = 4
    with chhs.Batch(runs, opts=chhs.default_opts(precision=1, max_inner=max_inner)) as b:
        for q, r in enumerate(runs):
            b.runs[q].set_phi(_phi0(r[0], q))
        st, vb, _ = b.step(nsteps)
        assert all(s == chhs.CHHS_OK for s in st)
        per_v, per_step = b.launch_counts()
        batched = [b.runs[q].get_state() for q in range(len(runs))]
    for q, (shape, h, eps, gamma, dt) in enumerate(runs):
        with chhs.Run(shape, h, eps, gamma, dt, opts=chhs.default_opts(precision=1, max_inner=max_inner)) as solo:
            solo.set_phi(_phi0(shape, q))
            _, vs, _ = solo.step(nsteps)
            ref = solo.get_state()
        assert vs == vb[q], (q, vs, vb[q])
        for a, c in zip(batched[q], ref):
            assert np.array_equal(a, c), q
    # one launch per kernel and level, whatever the number of runs
    assert per_v < 4 * 12 and per_step < 30, (per_v, per_step)


def test_batch_sampled_run_matches_oracle():
    runs = RUNS_2D[:4]
    with chhs.Batch(runs) as b:
        for q, r in enumerate(runs):
            b.runs[q].set_phi(_phi0(r[0], q))
        b.step(2)
        for q in (1, 3):
            shape, h, eps, gamma, dt = runs[q]
            phim, phimm1, mu, p = b.runs[q].get_state()
            b.step(1)
            gphi = b.runs[q].get_phi()
            o = oracle.step(phim, phimm1, oracle.Params(h, eps, gamma, dt, tol=1e-13, max_v=100),
                            2.0 * phim - phimm1, mu, p)
            assert o[5] == oracle.OK
            assert np.max(np.abs(gphi - o[0])) <= MIXED_TOL


def test_batch_mass_energy_through_member_handles():
    runs = RUNS_2D[:3]
    with chhs.Batch(runs) as b:
        for q, r in enumerate(runs):
            b.runs[q].set_phi(_phi0(r[0], q))
        m0 = [b.runs[q].mass() for q in range(3)]
        b.step(3)
        for q, (shape, h, eps, gamma, dt) in enumerate(runs):
            phim, phimm1, _, _ = b.runs[q].get_state()
            E, F = b.runs[q].energy()
            oE, oF = oracle.energy(phim, h, eps, phimm1)
            assert abs(E - oE) <= 1e-12 * max(1.0, abs(oE)) and abs(F - oF) <= 1e-12 * max(1.0, abs(oF))
            assert abs(b.runs[q].mass() - m0[q]) <= 3 * 1.1e-10 * np.prod(shape) * h * h
        # a member is stepped by its batch only
        with pytest.raises(chhs.ChhsError):
            b.runs[0].step(1)


def test_batch_reports_a_failed_run_and_advances_the_others():
    """Failure detection without a GPU fault: a NaN in one run's state makes
    that run's residual non-finite; it stops with CHHS_ERR_DIVERGED at its
    last accepted state, while the other run of the call advances exactly as
    it does alone."""
    runs = [((64, 64), 0.025, 0.05, 1.0, 0.005), ((64, 64), 0.025, 0.05, 1.0, 0.005)]
    good = _phi0((64, 64), 8)
    bad = _phi0((64, 64), 9)
    bad[10, 20] = np.nan
    with chhs.Batch(runs) as b:
        b.runs[0].set_phi(good)
        b.runs[1].set_phi(bad)
        st, v, r = b.step(2, check=False)
        assert st[0] == chhs.CHHS_OK
        assert st[1] == chhs.CHHS_ERR_DIVERGED
        phim, phimm1, _, _ = b.runs[1].get_state()
        assert np.array_equal(phim, bad, equal_nan=True) and np.array_equal(phimm1, bad, equal_nan=True)
        got = b.runs[0].get_phi()
        # the batch keeps working once the bad run has a valid state again
        b.runs[1].set_phi(good)
        st, _, _ = b.step(1)
        assert st == [chhs.CHHS_OK, chhs.CHHS_OK]
    with chhs.Run((64, 64), 0.025, 0.05, 1.0, 0.005, opts=chhs.default_opts(precision=1)) as solo:
        solo.set_phi(good)
        solo.step(2)
        assert np.array_equal(solo.get_phi(), got)


def test_full_batched_configuration_sampled_runs_match_oracle():
    """The batched configuration at its full size, as the bench runs it (256
    runs of 64^2 ... 1024^2, one chhs_batch, default options): after two
    steps, the third step of sampled runs -- the first run of each size,
    1024^2 included -- equals the oracle's step from the same state within
    the mixed-precision bound, and every run converged."""
    from paper_1611_02967_gb300 import experiments
    runs, phis, sizes = experiments.batched_runs(4, 256)
    sample = sorted({int(n): k for k, n in reversed(list(enumerate(sizes)))}.values())
    assert {int(sizes[k]) for k in sample} == {64, 128, 256, 512, 1024}
    with chhs.Batch(runs) as b:
        for k in range(len(runs)):
            b.runs[k].set_phi(phis[k])
        st, _, _ = b.step(2)
        assert all(x == chhs.CHHS_OK for x in st)
        before = {k: b.runs[k].get_state() for k in sample}
        st, v, r = b.step(1)
        assert all(x == chhs.CHHS_OK for x in st) and max(r) <= 1e-10
        after = {k: b.runs[k].get_phi() for k in sample}
    for k in sample:
        shape, h, eps, gamma, dt = runs[k]
        phim, phimm1, mu, p = before[k]
        o = oracle.step(phim, phimm1, oracle.Params(h, eps, gamma, dt, tol=1e-13, max_v=100),
                        2.0 * phim - phimm1, mu, p)
        assert o[5] == oracle.OK
        assert np.max(np.abs(after[k] - o[0])) <= MIXED_TOL, (k, shape)


@pytest.mark.parametrize("runs", [RUNS_2D[:4], RUNS_3D[:2]], ids=["2d", "3d"])
def test_batch_tuning_matches_solo_runs_with_the_same_tuning(runs):
    """chhs_batch_set_tuning: the batch with another tail size and one coarse
    sweep each way is bit-identical to solo runs given the same tuning."""
    tc = 256 if len(runs[0][0]) == 2 else 64
    with chhs.Batch(runs) as b:
        b.set_tuning(tc, 1, 1, tile=(32, 32, 512))  # the large levels' tiles: no effect on results
        for q, r in enumerate(runs):
            b.runs[q].set_phi(_phi0(r[0], q))
        st, vb, _ = b.step(3)
        assert all(s == chhs.CHHS_OK for s in st)
        batched = [b.runs[q].get_state() for q in range(len(runs))]
        with pytest.raises(chhs.ChhsError):
            b.set_tuning(tc, 0, 0)  # no sweep at all: refused, the setting kept
        st, _, _ = b.step(1)
        assert all(s == chhs.CHHS_OK for s in st)
    for q, (shape, h, eps, gamma, dt) in enumerate(runs):
        with chhs.Run(shape, h, eps, gamma, dt, opts=chhs.default_opts(precision=1)) as solo:
            solo.set_tuning(tc, 8192, 512, 1, 1, 32, 16, 3)
            solo.set_phi(_phi0(shape, q))
            _, vs, _ = solo.step(3)
            ref = solo.get_state()
        assert vs == vb[q]
        for a, c in zip(batched[q], ref):
            assert np.array_equal(a, c), q


def test_batch_autotune_keeps_every_state():
    runs = RUNS_2D[:4]
    with chhs.Batch(runs) as b:
        for q, r in enumerate(runs):
            b.runs[q].set_phi(_phi0(r[0], q))
        b.step(2)
        before = [b.runs[q].get_state() for q in range(len(runs))]
        t = b.autotune(2)
        assert t["tail_cells"] in (256, 1024, 4096) and (t["coarse_nu1"], t["coarse_nu2"]) in ((2, 2), (1, 1))
        assert t["tile"] in ((32, 16, 512), (32, 32, 512), (64, 16, 512))
        assert t["ms_per_step"] > 0
        after = [b.runs[q].get_state() for q in range(len(runs))]
        for x, y in zip(before, after):
            for u, w in zip(x, y):
                assert np.array_equal(u, w)
        st, _, r = b.step(2)
        assert all(s == chhs.CHHS_OK for s in st) and max(r) <= 1e-10


@pytest.mark.parametrize("tile", [(32, 16, 512), (32, 32, 512), (64, 16, 512)])
def test_batch_large_level_tile_shapes_match_solo_runs(tile):
    """A 512^2 run's finest level goes to its own tile launch inside the
    batch (with the tile shape of chhs_batch_set_tuning), the 64^2 run's to
    the batched launch: both stay bit-identical to solo runs."""
    runs = [((512, 512), 0.025, 0.05, 1.0, 0.005), ((64, 64), 0.025, 0.05, 2.0, 0.005)]
    with chhs.Batch(runs) as b:
        b.set_tuning(1024, 2, 2, tile=tile)
        for q, r in enumerate(runs):
            b.runs[q].set_phi(_phi0(r[0], q))
        st, vb, _ = b.step(2)
        assert all(s == chhs.CHHS_OK for s in st)
        batched = [b.runs[q].get_state() for q in range(len(runs))]
    for q, (shape, h, eps, gamma, dt) in enumerate(runs):
        with chhs.Run(shape, h, eps, gamma, dt, opts=chhs.default_opts(precision=1)) as solo:
            solo.set_phi(_phi0(shape, q))
            _, vs, _ = solo.step(2)
            ref = solo.get_state()
        assert vs == vb[q]
        for a, c in zip(batched[q], ref):
            assert np.array_equal(a, c), q
