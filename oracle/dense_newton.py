"""Dense Newton solve of one CHHS time step, for small grids only.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

This is a second, independent checker of ``chhs_oracle.c``: instead of
neighbour loops and multigrid it builds the Appendix A operators as explicit
matrices -- the face-to-centre difference d_x, the centre-to-face average A_x
and difference D_x, each a Kronecker product of a one-dimensional operator
with identities -- assembles the scheme (2.5)-(2.7) from them, and solves it
by Newton's method with a dense LU factorisation of the full 3N x 3N
Jacobian.  Homogeneous Neumann conditions enter exactly as Eq. A.1-A.3 say:
the ghost equals its neighbour, so D on a boundary face is zero.

The pressure is determined up to a constant (pure Neumann problem); one
pressure equation is redundant (the N3 rows sum to zero for any state), so
the last one is replaced by the gauge sum(p) = 0.
"""
import numpy as np


def _ops_1d(n, h):
    """(D, A, d) for one direction: faces 0..n (face k sits between cells k-1 and k)."""
    D = np.zeros((n + 1, n))
    A = np.zeros((n + 1, n))
    d = np.zeros((n, n + 1))
    for k in range(1, n):
        D[k, k - 1], D[k, k] = -1.0 / h, 1.0 / h
        A[k, k - 1], A[k, k] = 0.5, 0.5
    # boundary faces: ghost = mirror, so D = 0 and A = the adjacent cell value
    A[0, 0] = 1.0
    A[n, n - 1] = 1.0
    for c in range(n):
        d[c, c], d[c, c + 1] = -1.0 / h, 1.0 / h
    return D, A, d


def operators(shape, h):
    """Lists (D_a, A_a, d_a) over axes a = x, y (, z) for arrays indexed [.., y, x]."""
    dims = list(shape)[::-1]  # (nx, ny[, nz])
    ops = []
    for a, na in enumerate(dims):
        D1, A1, d1 = _ops_1d(na, h)
        mats = []
        for M1 in (D1, A1, d1):
            # kron over axes ordered slowest..fastest: z, y, x
            full = np.ones((1, 1))
            for b in reversed(range(len(dims))):
                full = np.kron(full, M1 if b == a else np.eye(dims[b]))
            mats.append(full)
        ops.append(tuple(mats))
    return ops


def solve_step(phim, phimm1, h, eps, gamma, s, tol=1e-14, max_iter=50, phi_guess=None):
    """Return (phi^{m+1}, mu, p) solving (2.5)-(2.7) to ||F||_inf <= tol."""
    shape = phim.shape
    pm = phim.ravel().astype(np.float64)
    pm1 = phimm1.ravel().astype(np.float64)
    N = pm.size
    ops = operators(shape, h)
    ps = 1.5 * pm - 0.5 * pm1                   # phi*  (Eq. 2.4)
    lap = sum(d @ D for D, A, d in ops)          # Delta_h = div_h grad_h
    # face operators weighted by A_h phi*
    divM = sum(d @ np.diag(1.0 + gamma * (A @ ps) ** 2) @ D for D, A, d in ops)
    diva = sum(d @ np.diag(A @ ps) @ D for D, A, d in ops)
    f_phi = pm
    f_mu = -ps - 0.25 * eps ** 2 * (lap @ pm1)
    I = np.eye(N)

    def F(z):
        phi, mu, p = z[:N], z[N:2 * N], z[2 * N:]
        chi = 0.25 * (phi ** 2 + pm ** 2) * (phi + pm)
        n1 = phi - s * (divM @ mu) - s * (diva @ p) - f_phi
        n2 = mu - chi + 0.75 * eps ** 2 * (lap @ phi) - f_mu
        n3 = -(lap @ p) - gamma * (diva @ mu)
        n3[-1] = p.sum()
        return np.concatenate([n1, n2, n3])

    def J(z):
        phi = z[:N]
        dchi = 0.25 * (3.0 * phi ** 2 + 2.0 * phi * pm + pm ** 2)
        top = np.hstack([I, -s * divM, -s * diva])
        mid = np.hstack([-np.diag(dchi) + 0.75 * eps ** 2 * lap, I, np.zeros((N, N))])
        bot = np.hstack([np.zeros((N, N)), -gamma * diva, -lap])
        Jm = np.vstack([top, mid, bot])
        Jm[-1, :] = 0.0
        Jm[-1, 2 * N:] = 1.0
        return Jm

    z = np.concatenate([pm if phi_guess is None else phi_guess.ravel(), np.zeros(2 * N)])
    for _ in range(max_iter):
        r = F(z)
        if np.max(np.abs(r)) <= tol:
            break
        z = z - np.linalg.solve(J(z), r)
    else:
        raise RuntimeError("dense Newton did not converge: %g" % np.max(np.abs(F(z))))
    return z[:N].reshape(shape), z[N:2 * N].reshape(shape), z[2 * N:].reshape(shape)
