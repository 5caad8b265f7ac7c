"""Pins of the oracle's face velocity (Eq. 2.3, u = -grad_h p - gamma A_h phi* grad_h mu)
against closed forms.  The face between cells i and i+1 is stored at i; boundary
faces carry zero normal velocity.  For a Neumann cosine mode the difference
quotient has the closed form  -(cos(k x_{i+1}) - cos(k x_i)) / h
= (2/h) sin(k x_{i+1/2}) sin(k h / 2), and the face average of a linear phi*
is its value at the face centre."""
import numpy as np

import oracle


def _centres(n, h):
    return (np.arange(n) + 0.5) * h


def _mode_quotient(n, h, L):
    xf = (np.arange(n) + 1.0) * h  # face centres x_{i+1/2}
    q = (2.0 / h) * np.sin(np.pi * xf / L) * np.sin(np.pi * h / (2.0 * L))
    q[-1] = 0.0  # boundary face
    return q, xf


def test_pressure_mode_gives_closed_form_velocity():
    nx, ny, h = 24, 16, 0.1
    L = nx * h
    x = _centres(nx, h)
    rng = np.random.default_rng(3)
    p = np.tile(np.cos(np.pi * x / L), (ny, 1))
    mu = rng.standard_normal((ny, nx))
    phis = rng.standard_normal((ny, nx))
    u = oracle.face_velocity(phis, mu, p, h, 0.0)  # gamma = 0: u = -grad_h p
    q, _ = _mode_quotient(nx, h, L)
    assert np.allclose(u[0], np.tile(q, (ny, 1)), rtol=0, atol=1e-12)
    assert np.array_equal(u[1], np.zeros((ny, nx)))


def test_mobility_term_with_linear_phi_star():
    nx, ny, h, gamma = 12, 20, 0.05, 2.5
    L = ny * h
    y = _centres(ny, h)
    mu = np.tile(np.cos(np.pi * y / L)[:, None], (1, nx))
    phis = np.tile(y[:, None], (1, nx))
    u = oracle.face_velocity(phis, mu, np.zeros((ny, nx)), h, gamma)
    q, yf = _mode_quotient(ny, h, L)
    expect = gamma * yf * q  # -gamma (A phi*) D mu with A phi* = y_{j+1/2}
    assert np.allclose(u[1], np.tile(expect[:, None], (1, nx)), rtol=0, atol=1e-12)
    assert np.array_equal(u[0], np.zeros((ny, nx)))


def test_3d_z_mode_and_norm_and_divergence():
    n, h = 8, 0.2
    L = n * h
    z = _centres(n, h)
    p = np.broadcast_to(np.cos(np.pi * z / L)[:, None, None], (n, n, n)).copy()
    rng = np.random.default_rng(5)
    phis = rng.standard_normal((n, n, n))
    u = oracle.face_velocity(phis, np.zeros((n, n, n)), p, h, 1.7)
    q, _ = _mode_quotient(n, h, L)
    assert np.allclose(u[2], np.broadcast_to(q[:, None, None], (n, n, n)), rtol=0, atol=1e-12)
    assert np.array_equal(u[0], np.zeros_like(p)) and np.array_equal(u[1], np.zeros_like(p))
    # the same faces through the norm and the divergence of oracle.velocity
    mu = rng.standard_normal((n, n, n))
    p = rng.standard_normal((n, n, n))
    u = oracle.face_velocity(phis, mu, p, h, 1.7)
    u2, div = oracle.velocity(phis, mu, p, h, 1.7)
    assert abs(h ** 3 * np.sum(u * u) - u2) <= 1e-12 * u2
    d = np.zeros_like(p)
    for a, ax in ((0, 2), (1, 1), (2, 0)):
        d += u[a] / h
        d -= np.roll(u[a], 1, axis=ax) / h  # face i-1/2 is stored at i-1 (zero at i = 0 below)
        first = [slice(None)] * 3
        first[ax] = 0
        d[tuple(first)] += np.roll(u[a], 1, axis=ax)[tuple(first)] / h
    assert np.allclose(d, div, rtol=0, atol=1e-10)
