"""V-cycles between stopping norms (chhs_opts.max_inner).

After each stopping norm the device predicts from the measured contraction
how many V-cycles the norm still needs and runs up to max_inner of them
before the next norm (graph IF nodes inside the step's loop).  The steps must
still end only on a norm at or below tol, so every step of a run with
max_inner = 4 must equal the oracle's step like the one-norm-per-V-cycle
run's, with fewer norms and no more than one extra V-cycle per step.
"""
import numpy as np
import pytest

import oracle
from paper_1611_02967_gb300 import chhs, inputs

pytestmark = pytest.mark.gpu

CASES = [  # (shape, h, eps, gamma, dt, precision, tol_phi, steps)
    ((256, 256), 0.025, 0.05, 1.0, 0.005, 0, 1e-9, 6),
    ((256, 256), 0.025, 0.05, 1.0, 0.005, 1, 1e-8, 6),
    ((32, 32, 32), 0.05, 0.04, 2.0, 0.005, 1, 1e-8, 4),
    ((24, 40), 0.1, 0.08, 0.0, 0.01, 0, 1e-9, 5),
]


@pytest.mark.parametrize("case", CASES, ids=lambda c: "x".join(map(str, c[0])) + "-p%d-g%g" % (c[5], c[3]))
def test_inner_vcycles_match_oracle_with_fewer_norms(case):
    shape, h, eps, gamma, dt, prec, tol_phi, steps = case
    phi0 = inputs.spinodal(shape, 7, mean=0.0) if len(shape) == 2 else \
        inputs.bubbles(shape[0], shape[0] * h, eps, 7, count=3)
    prm = oracle.Params(h, eps, gamma, dt, tol=1e-13, max_v=100)
    out = {}
    for mi in (1, 4):
        vs, checks, states = [], [], []
        with chhs.Run(shape, h, eps, gamma, dt, opts=chhs.default_opts(precision=prec, max_inner=mi)) as run:
            run.set_phi(phi0)
            for k in range(steps):
                before = run.get_state()
                _, v, r = run.step(1)
                assert r <= 1e-10
                vs.append(v)
                checks.append(run.norm_checks())
                phim, phimm1, mu, p = before
                o = oracle.step(phim, phimm1, prm, 2.0 * phim - phimm1, mu, p)
                assert o[5] == oracle.OK
                assert np.max(np.abs(run.get_phi() - o[0])) <= tol_phi, (mi, k)
                states.append(run.get_phi())
        out[mi] = (vs, checks, states)
    v1, c1, s1 = out[1]
    v3, c3, s3 = out[4]
    assert c1 == v1  # one norm per V-cycle
    assert sum(c3) < sum(c1)
    assert all(b <= a + 1 for a, b in zip(v1, v3)), (v1, v3)
    for a, b in zip(s1, s3):
        assert np.max(np.abs(a - b)) <= 2 * tol_phi


def test_eager_profile_step_follows_the_inner_counts():
    """The kernel-by-kernel step (chhs_profile_step) runs the same iterations
    as the graph: same V-cycles from the same state, and the same phi."""
    shape, h = (128, 128), 0.05
    phi0 = inputs.spinodal(shape, 3, mean=0.0)
    with chhs.Run(shape, h, 0.05, 1.0, 0.01, opts=chhs.default_opts(precision=1)) as a, \
            chhs.Run(shape, h, 0.05, 1.0, 0.01, opts=chhs.default_opts(precision=1)) as b:
        a.set_phi(phi0)
        b.set_phi(phi0)
        a.step(3)
        b.step(3)
        _, va, _ = a.step(1)
        acc = b.profile_step()
        assert np.max(np.abs(a.get_phi() - b.get_phi())) <= 1e-12
        assert a.norm_checks() < va or va <= 1


@pytest.mark.parametrize("precision", [0, 1])
def test_inner_vcycles_respect_max_v(precision):
    """The predicted V-cycles never take a step past max_v: a step capped
    below what it needs stops with CHHS_ERR_NOT_CONVERGED after exactly
    max_v V-cycles (the count of the one-norm-per-V-cycle run), state kept."""
    shape, h = (128, 128), 0.025
    phi0 = inputs.spinodal(shape, 5, mean=0.0)
    for max_v in (2, 4):
        with chhs.Run(shape, h, 0.05, 1.0, 0.005,
                      opts=chhs.default_opts(precision=precision, max_v=max_v, max_inner=4)) as run:
            run.set_phi(phi0)
            st, v, r = run.step(1, check=False)
            assert st == chhs.CHHS_ERR_NOT_CONVERGED
            assert v == max_v
            assert r > 1e-10
            phim, phimm1, _, _ = run.get_state()
            assert np.array_equal(phim, phi0) and np.array_equal(phimm1, phi0)
