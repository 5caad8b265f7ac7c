"""Pins of the oracle's time step against what Section 2 fixes.

- dense Newton agreement on grids of 16x16 and smaller (the step's solution
  is unique, Theorem 2.1), so the multigrid converges to the right answer;
- the exact discrete energy law behind Eq. 2.23 ("energy-est-15"): the two
  Cauchy inequalities of the proof become equalities once their slack
  1/4 ||a - b||^2 + 1/8 eps^2 ||grad(a - b)||^2 is added back, so with
  a = phi^{m+1} - phi^m and b = phi^m - phi^{m-1}
      F_h(phi^{m+1}, phi^m) - F_h(phi^m, phi^{m-1}) + slack
          + s ||grad mu||^2 + (s/gamma) ||u||^2 = 0
  up to the solver residual.  A dropped term, a wrong sign or a wrong
  coefficient anywhere in (2.5)-(2.7) breaks it;
- mass conservation (Section 4) within the residual bound;
- div_h u = 0 (Eq. 2.7);
- for data varying in x only, (2.7) forces u = 0 and the step does not
  depend on gamma (follows from 2.5-2.7 with M = 1 + gamma (A phi*)^2);
- reflection symmetry.
"""
import numpy as np
import pytest

import oracle
from oracle import dense_newton
from paper_1611_02967_gb300 import inputs


def _prm(h, eps, gamma, s, tol=1e-13):
    return oracle.Params(h, eps, gamma, s, tol=tol, max_v=100)


@pytest.mark.parametrize("shape,h,eps,gamma,s", [
    ((16, 16), 0.2, 0.1, 2.0, 0.02),
    ((8, 16), 0.2, 0.15, 1.0, 0.05),
    ((8, 8), 0.4, 0.2, 4.0, 0.1),
    ((4, 4, 4), 0.4, 0.1, 2.0, 0.02),
    ((2, 2), 0.5, 0.2, 1.0, 0.01),
    ((8, 16), 0.3, 0.15, 0.0, 0.05),
])
def test_fas_matches_dense_newton(shape, h, eps, gamma, s):
    phim = inputs.spinodal(shape, 11, mean=0.1, amplitude=0.6)
    phimm1 = inputs.spinodal(shape, 12, mean=0.1, amplitude=0.6)
    phi, mu, p, v, r, st = oracle.step(phim, phimm1, _prm(h, eps, gamma, s))
    assert st == oracle.OK
    dphi, dmu, dp = dense_newton.solve_step(phim, phimm1, h, eps, gamma, s)
    assert np.max(np.abs(phi - dphi)) < 1e-12
    assert np.max(np.abs(mu - dmu)) < 1e-12
    assert np.max(np.abs((p - p.mean()) - (dp - dp.mean()))) < 1e-11


def _energy_law_defect(phip, phim, phimm1, mu, p, h, eps, gamma, s):
    a = phip - phim
    b = phim - phimm1
    _, F1 = oracle.energy(phip, h, eps, phim)
    _, F0 = oracle.energy(phim, h, eps, phimm1)
    slack = 0.25 * oracle.inner(a - b, a - b, h) + 0.125 * eps ** 2 * oracle.grad_inner(a - b, a - b, h)
    gmu = oracle.grad_inner(mu, mu, h)
    u2, _ = oracle.velocity(1.5 * phim - 0.5 * phimm1, mu, p, h, gamma)
    # at gamma = 0 the pressure decouples (Eq. 2.7: Lap_h p = 0, p constant),
    # u = 0 and the law has no velocity term
    terms = (F1 - F0, slack, s * gmu, s / gamma * u2 if gamma > 0 else 0.0)
    return sum(terms), max(abs(t) for t in terms)


@pytest.mark.parametrize("shape,gamma", [((32, 32), 1.0), ((16, 16, 16), 2.0), ((32, 16), 0.0)])
def test_exact_discrete_energy_law(shape, gamma):
    n = shape[0]
    h = 3.2 / n
    eps, s = 0.1, 0.01
    phi0 = inputs.spinodal(shape, 21, mean=0.0, amplitude=0.4)
    prm = _prm(h, eps, gamma, s)
    defects = []

    def cb(k, phi, phim, phimm1, mu, p):
        d, scale = _energy_law_defect(phi, phim, phimm1, mu, p, h, eps, gamma, s)
        defects.append((d, scale))
        if gamma == 0.0:
            assert np.max(np.abs(p)) < 1e-12  # mean-free constant

    oracle.run(phi0, prm, 6, callback=cb)
    for d, scale in defects:
        assert abs(d) < 1e-12 * max(scale, 1.0), defects


def test_energy_law_detects_wrong_scheme():
    # Sensitivity of the pin: the solution of a different scheme (phi^{m-1}
    # replaced by phi^m inside the solve, i.e. first-order phi* and no
    # 1/4 eps^2 Lap phi^{m-1} term) violates the law by far more than the
    # tolerance above.
    shape, h, eps, gamma, s = (32, 32), 0.1, 0.1, 1.0, 0.01
    phi0 = inputs.spinodal(shape, 21, mean=0.0, amplitude=0.4)
    prm = _prm(h, eps, gamma, s)
    phim, phimm1, mu, p, _ = oracle.run(phi0, prm, 3)
    wrong, mu_w, p_w, _, _, st = oracle.step(phim, phim, prm)
    assert st == oracle.OK
    d, scale = _energy_law_defect(wrong, phim, phimm1, mu_w, p_w, h, eps, gamma, s)
    assert abs(d) > 1e-6 * scale


@pytest.mark.parametrize("s", [0.08, 0.04, 0.02, 0.01, 0.005])
def test_modified_energy_non_increasing_every_dt(s):
    # Eq. 2.23: F_h(phi^{m+1}, phi^m) <= F_h(phi^m, phi^{m-1}) for any s > 0.
    shape, h, eps, gamma = (32, 32), 0.1, 0.05, 2.0
    phi0 = inputs.spinodal(shape, 31, mean=-0.05, amplitude=0.05)
    prm = _prm(h, eps, gamma, s, tol=1e-12)
    F = []

    def cb(k, phi, phim, phimm1, mu, p):
        if k == 0:
            F.append(oracle.energy(phim, h, eps, phimm1)[1])
        F.append(oracle.energy(phi, h, eps, phim)[1])

    oracle.run(phi0, prm, 12, callback=cb)
    assert all(F[k + 1] <= F[k] + 1e-12 for k in range(len(F) - 1)), F


def test_mass_conserved_within_residual_bound():
    # (phi^{m+1}, 1) - (phi^m, 1) = -h^d sum r_phi, |h^d sum r_phi| <= |Omega| ||r||
    w = inputs.workload("spinodal64")
    h = w["h"]
    area = 64 * 64 * h * h
    prm = oracle.Params(h, w["eps"], w["gamma"], w["dt"], tol=1e-10)
    m0 = oracle.mass(w["phi0"], h)
    drift = []

    def cb(k, phi, phim, phimm1, mu, p):
        drift.append(abs(oracle.mass(phi, h) - oracle.mass(phim, h)))

    oracle.run(w["phi0"], prm, 10, callback=cb)
    bound = area * 1e-10 + 1e-13 * area
    assert max(drift) <= bound
    assert abs(m0 - (-0.05) * area) < 0.05 * area * 0.02


def test_divergence_free_velocity():
    shape, h, eps, gamma, s = (32, 32), 0.1, 0.1, 2.0, 0.01
    phi0 = inputs.spinodal(shape, 41, mean=0.0, amplitude=0.5)
    checks = []

    def cb(k, phi, phim, phimm1, mu, p):
        # u of Eq. 2.3 uses the phi* of this step
        checks.append(oracle.velocity(1.5 * phim - 0.5 * phimm1, mu, p, h, gamma))

    oracle.run(phi0, _prm(h, eps, gamma, s), 3, callback=cb)
    for u2, div in checks:
        assert u2 > 1e-8  # the flow is not trivially zero
        assert np.max(np.abs(div)) < 1e-9


def test_x_only_data_is_gamma_independent():
    # For phi varying in x only, (2.7) gives D_x p = -gamma A_x phi* D_x mu,
    # so u = 0 and (2.5) reduces to phi - s Lap_h mu: the step is the pure
    # Cahn-Hilliard step for every gamma.
    nx, ny, h = 32, 8, 0.1
    x = (np.arange(nx) + 0.5) * h
    row = 0.6 * np.cos(np.pi * x / (nx * h)) + 0.2 * np.cos(3 * np.pi * x / (nx * h))
    phim = np.tile(row, (ny, 1))
    phimm1 = np.tile(0.98 * row, (ny, 1))
    res = []
    for gamma in (0.0, 1.0, 4.0):
        phi, mu, p, v, r, st = oracle.step(phim, phimm1, _prm(h, 0.1, gamma, 0.02))
        assert st == oracle.OK
        res.append((phi, mu))
        u2, _ = oracle.velocity(1.5 * phim - 0.5 * phimm1, mu, p, h, gamma)
        assert u2 < 1e-20
    for phi, mu in res[1:]:
        assert np.max(np.abs(phi - res[0][0])) < 1e-12
        assert np.max(np.abs(mu - res[0][1])) < 1e-12


def test_reflection_symmetry():
    shape, h, eps, gamma, s = (16, 32), 0.1, 0.08, 2.0, 0.02
    phim = inputs.spinodal(shape, 51, mean=0.0, amplitude=0.5)
    phimm1 = inputs.spinodal(shape, 52, mean=0.0, amplitude=0.5)
    prm = _prm(h, eps, gamma, s)
    a = oracle.step(phim, phimm1, prm)[0]
    b = oracle.step(phim[:, ::-1], phimm1[:, ::-1], prm)[0][:, ::-1]
    c = oracle.step(phim[::-1, :], phimm1[::-1, :], prm)[0][::-1, :]
    assert np.max(np.abs(a - b)) < 1e-12 and np.max(np.abs(a - c)) < 1e-12


def test_status_codes():
    shape = (16, 16)
    phim = inputs.spinodal(shape, 61, mean=0.0, amplitude=0.5)
    prm = oracle.Params(0.1, 0.05, 1.0, 0.01, tol=1e-10, max_v=1)
    st = oracle.step(phim, phim, prm)[5]
    assert st == oracle.NOT_CONVERGED
    bad = oracle.Params(-0.1, 0.05, 1.0, 0.01)
    assert oracle.step(phim, phim, bad)[5] == oracle.BAD_ARG
