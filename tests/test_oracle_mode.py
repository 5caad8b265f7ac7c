"""Closed-form pin of the oracle's time step: one small cosine mode.

Take phi^{m-1} = pbar + a_{m-1} v and phi^m = pbar + a_m v, with v one
cosine mode of the cell-centred Neumann grid, so Lap_h v = -lam v, where
lam = sum over directions of (4/h^2) sin^2(pi k / (2n)).  Linearise
Eqs. 2.5-2.7 about the constant pbar (A_h phi* = pbar at first order):

- Eq. 2.7 gives -lam p = gamma pbar lam mu for the mode amplitudes, so
  p = -gamma pbar mu;
- in Eq. 2.5 the mobility term s (1 + gamma pbar^2)(-lam) mu and the
  pressure term s pbar (-lam) p add to -s lam mu: the step does not depend
  on gamma;
- Eq. 2.6 with chi(a, b) = (a^2 + b^2)(a + b)/4, whose partial derivatives
  at (pbar, pbar) are both 3 pbar^2 / 2, and phi* = 3/2 phi^m - 1/2 phi^{m-1}
  (Eq. 2.4), gives
      mu = 3/2 pbar^2 (a_{m+1} + a_m) - (3/2 a_m - 1/2 a_{m-1})
           + eps^2 lam (3/4 a_{m+1} + 1/4 a_{m-1}).

Eliminating mu:

    a_{m+1} (1 + s lam (3/2 pbar^2 + 3/4 eps^2 lam))
        = a_m (1 - s lam (3/2 pbar^2 - 3/2)) - a_{m-1} s lam (1/2 + 1/4 eps^2 lam).

The mean of mu is chi(pbar, pbar) - pbar = pbar^3 - pbar.  The neglected
terms are products of two copies of the mode: their Fourier content is the
constant and the doubled frequencies, orthogonal to v, so the projection of
the solution on v is exact up to O(a^3), i.e. relative O(a^2).  A wrong
weight, sign, splitting or Laplacian scale in the oracle moves a_{m+1}, mu
or p by a relative 1e-3 or more; the tolerances below are 1e-8.
"""
import numpy as np
import pytest

import oracle


def _mode(shape, ks):
    # numpy order (z, y, x) / (y, x); ks in the same order
    v = np.ones(shape)
    for ax, k in enumerate(ks):
        n = shape[ax]
        c = np.cos(np.pi * k * (np.arange(n) + 0.5) / n)
        sh = [1] * len(shape)
        sh[ax] = n
        v = v * c.reshape(sh)
    return v


def _lam(shape, ks, h):
    return sum(4.0 / h ** 2 * np.sin(np.pi * k / (2 * n)) ** 2 for n, k in zip(shape, ks))


def _closed(a0, am1, pbar, eps, s, lam, w34=0.75, w14=0.25, c_star=(1.5, -0.5), d1=1.5, d0=1.5):
    """a_{m+1}, mu amplitude of the linearised step.  The keyword arguments
    exist only so that the sensitivity test can evaluate wrong variants."""
    q = pbar ** 2
    star = c_star[0] * a0 + c_star[1] * am1
    lhs = 1.0 + s * lam * (d1 * q + w34 * eps ** 2 * lam)
    rhs = a0 - s * lam * (d0 * q * a0 - star + w14 * eps ** 2 * lam * am1)
    a1 = rhs / lhs
    mu = d1 * q * a1 + d0 * q * a0 - star + eps ** 2 * lam * (w34 * a1 + w14 * am1)
    return a1, mu


CASES = [
    # shape, mode numbers, h, eps, gamma, s, pbar
    ((24, 32), (2, 3), 0.1, 0.1, 2.0, 0.02, 0.3),
    ((24, 32), (1, 0), 0.1, 0.05, 0.0, 0.05, -0.4),
    ((32, 16), (5, 2), 0.2, 0.15, 4.0, 0.01, 0.0),
    ((8, 16, 8), (1, 3, 2), 0.2, 0.15, 1.5, 0.03, -0.2),
]
DELTA = 1e-5


def _solve(shape, ks, h, eps, gamma, s, pbar):
    v = _mode(shape, ks)
    a0, am1 = DELTA, 0.9 * DELTA
    phi, mu, p, nv, r, st = oracle.step(pbar + a0 * v, pbar + am1 * v,
                                        oracle.Params(h, eps, gamma, s, tol=1e-14, max_v=200))
    assert st == oracle.OK

    def proj(f):
        return float(np.sum(f * v) / np.sum(v * v))

    return v, a0, am1, phi, mu, p, proj


@pytest.mark.parametrize("case", range(len(CASES)))
def test_single_mode_step_matches_linearised_scheme(case):
    shape, ks, h, eps, gamma, s, pbar = CASES[case]
    v, a0, am1, phi, mu, p, proj = _solve(*CASES[case])
    lam = _lam(shape, ks, h)
    a1c, muc = _closed(a0, am1, pbar, eps, s, lam)
    assert abs(proj(phi - pbar) - a1c) < 1e-8 * DELTA
    assert abs(proj(mu) - muc) < 1e-8 * max(abs(muc), DELTA)
    assert abs(mu.mean() - (pbar ** 3 - pbar)) < 1e-8
    assert abs(proj(p - p.mean()) - (-gamma * pbar * muc)) < 1e-8 * max(abs(gamma * pbar * muc), DELTA)
    # mass exactly conserved; the rest of the solution is the O(a^2) harmonics
    assert abs(phi.mean() - pbar) < 1e-14
    assert np.max(np.abs(phi - pbar - proj(phi - pbar) * v)) < 1e-3 * DELTA


WRONG = {
    "3/4 and 1/4 of the eps^2 term swapped": dict(w34=0.25, w14=0.75),
    "first-order phi* = phi^m": dict(c_star=(1.0, 0.0)),
    "phi* weights reversed": dict(c_star=(-0.5, 1.5)),
    "fully implicit cubic": dict(d1=3.0, d0=0.0),
    "explicit cubic": dict(d1=0.0, d0=3.0),
    "phi* term with the wrong sign": dict(c_star=(-1.5, 0.5)),
}


@pytest.mark.parametrize("case", [0, 3])
def test_pin_separates_plausible_wrong_schemes(case):
    # each wrong variant of the scheme predicts an a_{m+1} or mu that the
    # oracle's solution misses by far more than the tolerance above
    shape, ks, h, eps, gamma, s, pbar = CASES[case]
    v, a0, am1, phi, mu, p, proj = _solve(*CASES[case])
    lam = _lam(shape, ks, h)
    a1, m1 = proj(phi - pbar), proj(mu)
    for name, kw in WRONG.items():
        a1w, muw = _closed(a0, am1, pbar, eps, s, lam, **kw)
        miss = max(abs(a1 - a1w) / DELTA, abs(m1 - muw) / max(abs(muw), DELTA))
        assert miss > 1e-4, name
    # and the Laplacian scale: 1/h in place of 1/h^2
    a1w, _ = _closed(a0, am1, pbar, eps, s, lam * h)
    assert abs(a1 - a1w) > 1e-4 * DELTA
