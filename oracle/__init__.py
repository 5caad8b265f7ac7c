"""CPU oracle for the CHHS time step (Section 2, Eqs. 2.4-2.7).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` may import this package.  It shares no
code with the CUDA library (``paper_1611_02967_gb300``) and neither imports
the other; the seeded input generators in ``paper_1611_02967_gb300.inputs``
hold none of the method's arithmetic and are the only thing both sides use.

``chhs_oracle.c`` is a plain double-precision lexicographic nonlinear
Gauss-Seidel FAS solver of the implicit system (2.5)-(2.7); ``dense_newton``
solves the same system by a dense Newton method built from the Appendix A
operator definitions, as an independent check of the multigrid.
"""
import ctypes
import os

import numpy as np

from . import build as _build

_lib = None

OK, NOT_CONVERGED, DIVERGED, BAD_ARG, OOM = 0, 1, 2, 3, 4

_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int)


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        d, i = ctypes.c_double, ctypes.c_int
        L.oracle_step.argtypes = [i, _ip, d, d, d, d, _dp, _dp, _dp, _dp, _dp,
                                  i, i, i, d, i, _ip, _dp]
        L.oracle_step.restype = i
        L.oracle_residual.argtypes = [i, _ip, d, d, d, d, _dp, _dp, _dp, _dp, _dp, _dp, _dp, _dp]
        L.oracle_residual.restype = d
        L.oracle_laplacian.argtypes = [i, _ip, d, _dp, _dp]
        L.oracle_laplacian.restype = None
        L.oracle_inner.argtypes = [i, _ip, d, _dp, _dp]
        L.oracle_inner.restype = d
        L.oracle_grad_inner.argtypes = [i, _ip, d, _dp, _dp]
        L.oracle_grad_inner.restype = d
        L.oracle_mass.argtypes = [i, _ip, d, _dp]
        L.oracle_mass.restype = d
        L.oracle_energy.argtypes = [i, _ip, d, d, _dp, _dp, _dp, _dp]
        L.oracle_energy.restype = None
        L.oracle_velocity.argtypes = [i, _ip, d, d, _dp, _dp, _dp, _dp, _dp]
        L.oracle_velocity.restype = d
        L.oracle_num_levels.argtypes = [i, _ip, i]
        L.oracle_num_levels.restype = i
        _lib = L
    return _lib


def _f64(a):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a


def _ptr(a):
    return a.ctypes.data_as(_dp) if a is not None else None


def _dims(shape):
    """Arrays are indexed [z][y][x] (x fastest in memory); the C side wants (nx, ny, nz)."""
    n = list(shape[::-1]) + [1] * (3 - len(shape))
    return len(shape), (ctypes.c_int * 3)(*n)


class Params:
    """Physical and solver parameters of one run (Section 2 and Section 5)."""

    def __init__(self, h, eps, gamma, dt, nu1=2, nu2=2, max_v=60, tol=1e-10, coarsest=2):
        self.h, self.eps, self.gamma, self.dt = float(h), float(eps), float(gamma), float(dt)
        self.nu1, self.nu2, self.max_v, self.tol, self.coarsest = nu1, nu2, max_v, tol, coarsest


def step(phim, phimm1, prm, phi=None, mu=None, p=None):
    """Solve one time step from (phi^m, phi^{m-1}).

    Returns (phi^{m+1}, mu^{m+1/2}, p^{m+1/2}, vcycles, residual, status).
    The initial guess is phi = phi^m unless given, mu and p zero unless given.
    """
    phim, phimm1 = _f64(phim), _f64(phimm1)
    dim, n = _dims(phim.shape)
    phi = _f64(phim).copy() if phi is None else _f64(phi).copy()
    mu = np.zeros_like(phim) if mu is None else _f64(mu).copy()
    p = np.zeros_like(phim) if p is None else _f64(p).copy()
    v = ctypes.c_int(0)
    r = ctypes.c_double(0.0)
    st = lib().oracle_step(dim, n, prm.h, prm.eps, prm.gamma, prm.dt, _ptr(phim), _ptr(phimm1),
                           _ptr(phi), _ptr(mu), _ptr(p), prm.nu1, prm.nu2, prm.max_v, prm.tol,
                           prm.coarsest, ctypes.byref(v), ctypes.byref(r))
    return phi, mu, p, v.value, r.value, st


def residual(phim, phimm1, phi, mu, p, prm):
    """(r_phi, r_mu, r_p, norm) with r = f - N(u) on the given grid."""
    phim, phimm1, phi, mu, p = map(_f64, (phim, phimm1, phi, mu, p))
    dim, n = _dims(phim.shape)
    rphi, rmu, rp = (np.empty_like(phim) for _ in range(3))
    nrm = lib().oracle_residual(dim, n, prm.h, prm.eps, prm.gamma, prm.dt, _ptr(phim), _ptr(phimm1),
                                _ptr(phi), _ptr(mu), _ptr(p), _ptr(rphi), _ptr(rmu), _ptr(rp))
    return rphi, rmu, rp, nrm


def laplacian(v, h):
    v = _f64(v)
    dim, n = _dims(v.shape)
    out = np.empty_like(v)
    lib().oracle_laplacian(dim, n, float(h), _ptr(v), _ptr(out))
    return out


def inner(f, g, h):
    f, g = _f64(f), _f64(g)
    dim, n = _dims(f.shape)
    return lib().oracle_inner(dim, n, float(h), _ptr(f), _ptr(g))


def grad_inner(f, g, h):
    f, g = _f64(f), _f64(g)
    dim, n = _dims(f.shape)
    return lib().oracle_grad_inner(dim, n, float(h), _ptr(f), _ptr(g))


def mass(phi, h):
    phi = _f64(phi)
    dim, n = _dims(phi.shape)
    return lib().oracle_mass(dim, n, float(h), _ptr(phi))


def energy(phi, h, eps, psi=None):
    """(E_h(phi), F_h(phi, psi)) of Eqs. 2.8-2.9; F is None without psi."""
    phi = _f64(phi)
    dim, n = _dims(phi.shape)
    E = ctypes.c_double(0.0)
    F = ctypes.c_double(0.0)
    psi_a = _f64(psi) if psi is not None else None
    lib().oracle_energy(dim, n, float(h), float(eps), _ptr(phi), _ptr(psi_a), ctypes.byref(E),
                        ctypes.byref(F) if psi is not None else None)
    return E.value, (F.value if psi is not None else None)


def velocity(phis, mu, p, h, gamma):
    """(||u||_2^2, div_h u) for u = -grad_h p - gamma A_h phi* grad_h mu (Eq. 2.3)."""
    phis, mu, p = map(_f64, (phis, mu, p))
    dim, n = _dims(phis.shape)
    div = np.empty_like(phis)
    u2 = lib().oracle_velocity(dim, n, float(h), float(gamma), _ptr(phis), _ptr(mu), _ptr(p), _ptr(div), None)
    return u2, div


def face_velocity(phis, mu, p, h, gamma):
    """The velocity of Eq. 2.3 on the face grid: array (dim,) + shape whose
    [a][c] entry is the a-component on the face between cell c and its +a
    neighbour (0 on boundary faces)."""
    phis, mu, p = map(_f64, (phis, mu, p))
    dim, n = _dims(phis.shape)
    faces = np.zeros((dim,) + phis.shape)
    lib().oracle_velocity(dim, n, float(h), float(gamma), _ptr(phis), _ptr(mu), _ptr(p), None, _ptr(faces))
    return faces


def num_levels(shape, coarsest=2):
    dim, n = _dims(tuple(shape))
    return lib().oracle_num_levels(dim, n, coarsest)


def run(phi0, prm, nsteps, phi_prev=None, callback=None):
    """Advance nsteps from phi^0 with phi^{-1} = phi^0 (Remark 2.2) unless given.

    The initial guess of each step is the linear extrapolation
    2 phi^m - phi^{m-1} for phi and the previous step's mu and p.  Returns (phi^{nsteps}, phi^{nsteps-1}, mu, p, list of V-cycle counts).
    """
    phim = _f64(phi0).copy()
    phimm1 = phim.copy() if phi_prev is None else _f64(phi_prev).copy()
    mu = np.zeros_like(phim)
    p = np.zeros_like(phim)
    counts = []
    for k in range(nsteps):
        phi, mu, p, v, r, st = step(phim, phimm1, prm, 2.0 * phim - phimm1, mu, p)
        if st != OK:
            raise RuntimeError("oracle step %d failed: status %d, residual %g" % (k, st, r))
        counts.append(v)
        if callback is not None:
            callback(k, phi, phim, phimm1, mu, p)
        phimm1, phim = phim, phi
    return phim, phimm1, mu, p, counts
