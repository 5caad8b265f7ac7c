"""Pins of the oracle's discrete operators against closed forms (Appendix A).

These tests check ``oracle/`` against what the mathematics fixes, not
against itself: Neumann cosine modes are exact eigenvectors of Delta_h,
summation by parts (Eq. A "summation-1") relates two separately coded sums,
and the energies of constant and cosine states have closed forms.
"""
import numpy as np
import pytest

import oracle
from oracle import dense_newton
from paper_1611_02967_gb300 import inputs


def _cos_mode(shape, h, ks):
    """prod_a cos(k_a pi x_a / L_a) at the cell centres x = (i + 1/2) h."""
    v = np.ones(shape)
    for axis, (n, k) in enumerate(zip(shape, ks)):
        x = (np.arange(n) + 0.5) * h
        L = n * h
        s = [1] * len(shape)
        s[axis] = n
        v = v * np.cos(k * np.pi * x / L).reshape(s)
    return v


@pytest.mark.parametrize("shape,ks", [((16, 24), (3, 5)), ((8, 8), (0, 7)), ((6, 8, 10), (1, 2, 3)),
                                      ((4, 4, 4), (3, 0, 1))])
def test_laplacian_neumann_eigenvector(shape, ks):
    # On the midpoint grid the mirror ghost of Eq. A.1-A.3 equals the cosine's
    # own value at -h/2, so Delta_h cos(k pi x/L) = -(4/h^2) sin^2(k pi h/(2L)) cos(.)
    h = 0.17
    v = _cos_mode(shape, h, ks)
    lam = 0.0
    for n, k in zip(shape, ks):
        lam -= 4.0 / h ** 2 * np.sin(k * np.pi * h / (2.0 * n * h)) ** 2
    out = oracle.laplacian(v, h)
    assert np.max(np.abs(out - lam * v)) < 1e-12 * max(1.0, abs(lam))


@pytest.mark.parametrize("shape", [(12, 20), (5, 6, 7)])
def test_summation_by_parts(shape):
    # (phi, Delta_h psi) = -(grad_h phi, grad_h psi) when psi is Neumann (Eq. A summation-1)
    h = 0.3
    phi = inputs.spinodal(shape, 5, mean=0.2, amplitude=1.0)
    psi = inputs.spinodal(shape, 6, mean=-0.1, amplitude=1.0)
    lhs = oracle.inner(phi, oracle.laplacian(psi, h), h)
    rhs = -oracle.grad_inner(phi, psi, h)
    assert abs(lhs - rhs) < 1e-12 * (abs(lhs) + 1.0)


def test_grad_norm_of_cosine_mode():
    # ||grad_h v||^2 = -(v, Delta_h v) = (4/h^2) sin^2(k pi h / 2L) ||v||^2
    shape, h, ks = (32, 16), 0.1, (5, 0)
    v = _cos_mode(shape, h, ks)
    lam = 4.0 / h ** 2 * np.sin(ks[0] * np.pi * h / (2.0 * shape[0] * h)) ** 2
    g2 = oracle.grad_inner(v, v, h)
    assert abs(g2 - lam * oracle.inner(v, v, h)) < 1e-12 * g2


def test_energy_closed_forms():
    shape, h, eps = (10, 14), 0.2, 0.3
    area = shape[0] * shape[1] * h * h
    c = 0.7
    E, F = oracle.energy(np.full(shape, c), h, eps, np.full(shape, c))
    expect = area * (0.25 * c ** 4 - 0.5 * c ** 2)  # Eq. 2.8 with grad = 0
    assert abs(E - expect) < 1e-13 and abs(F - expect) < 1e-13
    # F_h(phi, psi) - E_h(phi) = 1/4 ||phi - psi||^2 for a constant shift (Eq. 2.9)
    E1, F1 = oracle.energy(np.full(shape, c), h, eps, np.full(shape, c - 0.5))
    assert abs(F1 - E1 - 0.25 * 0.25 * area) < 1e-13
    assert abs(oracle.mass(np.full(shape, c), h) - c * area) < 1e-13


def test_chi_fixed_point_constant_state():
    # chi(c, c) = c^3 (Eq. 2.4): a constant state is an exact fixed point of a
    # step with mu = c^3 - c and p constant.
    shape, h = (16, 16), 0.1
    for c in (-0.9, 0.0, 0.35, 1.2):
        phim = np.full(shape, c)
        prm = oracle.Params(h, 0.05, 2.0, 0.01, tol=1e-13)
        phi, mu, p, v, r, st = oracle.step(phim, phim, prm)
        assert st == oracle.OK
        # starting from mu = 0 the solve stops at tol 1e-13 (cell-RMS residual)
        assert np.max(np.abs(phi - c)) < 1e-11
        assert np.max(np.abs(mu - (c ** 3 - c))) < 1e-11
        assert np.max(np.abs(p)) < 1e-11


def test_dense_operators_match_closed_form():
    # The dense checker's matrices also reproduce the Neumann eigenvalue, so
    # both checkers are pinned to the same closed form, not to each other.
    shape, h, ks = (6, 10), 0.25, (2, 3)
    v = _cos_mode(shape, h, ks)
    ops = dense_newton.operators(shape, h)
    lap = sum(d @ D for D, A, d in ops)
    lam = sum(-4.0 / h ** 2 * np.sin(k * np.pi / (2.0 * n)) ** 2 for n, k in zip(shape, ks))
    assert np.max(np.abs(lap @ v.ravel() - lam * v.ravel())) < 1e-11
