"""Seeded synthetic inputs shared by the CUDA path, the oracle and the tests.

This module holds none of the method's arithmetic: it only draws initial
fields.  Random numbers come from SplitMix64 (Steele, Lea and Flood, "Fast
splittable pseudorandom number generators", OOPSLA 2014) keyed by
(seed, cell index), so that every side sees bit-identical double inputs.

Arrays are numpy float64, indexed [y, x] in 2D and [z, y, x] in 3D (x fastest
in memory); cell (i, j, k) sits at ((i + 1/2) h, (j + 1/2) h, (k + 1/2) h),
the cell-centred points of Appendix A.1.
"""
import numpy as np

_M64 = (1 << 64) - 1


def _splitmix64(x):
    """SplitMix64 finaliser applied elementwise to a uint64 array (wrapping arithmetic)."""
    with np.errstate(over="ignore"):
        z = x + np.uint64(0x9E3779B97F4A7C15)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        return z ^ (z >> np.uint64(31))


def uniform01(seed, count, stream=0):
    """count doubles in [0, 1): the top 53 bits of SplitMix64(seed-key + index)."""
    key = np.uint64((seed * 0x632BE59BD9B4E019 + stream * 0x8CB92BA72F3D8DD7 + 1) & _M64)
    with np.errstate(over="ignore"):
        idx = np.arange(count, dtype=np.uint64) * np.uint64(0x9E3779B97F4A7C15) + key
    z = _splitmix64(idx)
    return (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def spinodal(shape, seed, mean=-0.05, amplitude=0.05):
    """phi0 = mean + amplitude * (2 r - 1), r ~ U[0,1) per cell (Section 5.2 recipe)."""
    n = int(np.prod(shape))
    r = uniform01(seed, n)
    return (mean + amplitude * (2.0 * r - 1.0)).reshape(shape)


def cosine_bump(n, L):
    """Eq. 5.1 on (0,L)^2: ([1 - cos(4 pi x/L)][1 - cos(2 pi y/L)])/2 - 1 at cell centres."""
    h = L / n
    x = (np.arange(n) + 0.5) * h
    X = x[None, :]
    Y = x[:, None]
    return (1.0 - np.cos(4.0 * np.pi * X / L)) * (1.0 - np.cos(2.0 * np.pi * Y / L)) / 2.0 - 1.0


def cosine_bump3(n, L):
    """A 3D analogue of Eq. 5.1 on (0,L)^3 (the paper's test is 2D only):
    ([1 - cos(4 pi x/L)][1 - cos(2 pi y/L)][1 - cos(2 pi z/L)])/4 - 1 at cell
    centres, shape (z, y, x); values in [-1, 1], mean -3/4."""
    h = L / n
    x = (np.arange(n) + 0.5) * h
    Z, Y, X = np.meshgrid(x, x, x, indexing="ij")
    return ((1.0 - np.cos(4.0 * np.pi * X / L)) * (1.0 - np.cos(2.0 * np.pi * Y / L))
            * (1.0 - np.cos(2.0 * np.pi * Z / L)) / 4.0 - 1.0)


def bubbles(n, L, eps, seed, count=8, rmin=0.5, rmax=1.0):
    """3D tanh bubbles on a phi = -1 background.

    Radii R_k ~ U(rmin, rmax); centres c_k ~ U over [R_k, L - R_k]^3 from the
    seed; phi0 = max_k tanh((R_k - |x - c_k|) / (sqrt(2) eps)), which is -1 far
    from every bubble and stays in [-1, 1] where bubbles overlap.
    """
    u = uniform01(seed, count * 4, stream=7).reshape(count, 4)
    R = rmin + (rmax - rmin) * u[:, 0]
    C = R[:, None] + (L - 2.0 * R[:, None]) * u[:, 1:4]
    h = L / n
    x = (np.arange(n) + 0.5) * h
    Z, Y, X = np.meshgrid(x, x, x, indexing="ij")
    phi = np.full((n, n, n), -1.0)
    for k in range(count):
        d = np.sqrt((X - C[k, 0]) ** 2 + (Y - C[k, 1]) ** 2 + (Z - C[k, 2]) ** 2)
        phi = np.maximum(phi, np.tanh((R[k] - d) / (np.sqrt(2.0) * eps)))
    return phi


# Named workloads: (shape, h, eps, gamma, dt, steps, initial-field recipe).
def workload(name):
    if name == "spinodal64":
        shape, L = (64, 64), 3.2
        return dict(shape=shape, h=L / 64, eps=0.05, gamma=1.0, dt=0.01, steps=50,
                    phi0=spinodal(shape, seed=1))
    if name == "spinodal512":
        shape, L = (512, 512), 12.8
        return dict(shape=shape, h=L / 512, eps=0.05, gamma=1.0, dt=0.005, steps=200,
                    phi0=spinodal(shape, seed=2, mean=0.0))
    if name == "bubbles128":
        L = 6.4
        return dict(shape=(128, 128, 128), h=L / 128, eps=0.04, gamma=2.0, dt=0.005, steps=100,
                    phi0=bubbles(128, L, 0.04, seed=3))
    if name == "bubbles256":  # the largest 3D grid of the serving configuration, same h
        L = 12.8
        return dict(shape=(256, 256, 256), h=L / 256, eps=0.04, gamma=2.0, dt=0.005, steps=10,
                    phi0=bubbles(256, L, 0.04, seed=3))
    raise KeyError(name)
