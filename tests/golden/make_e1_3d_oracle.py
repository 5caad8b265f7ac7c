"""Write tests/golden/e1_3d_oracle.txt: the CPU oracle's Cauchy differences
for a 3D version of the Table 1 setting of Section 5.1 (the 3D analogue of
Eq. 5.1 in inputs.cosine_bump3 on (0,3.2)^3, eps 0.2, gamma 2, s = 0.05 h,
T = 0.8, tol 1e-10), fine grids 16^3, 32^3 and 64^3.

Calls only oracle/ (and the seedless initial-data generator).  The Cauchy
difference uses cell-centred trilinear interpolation with mirrored ghosts and
the h_f^3-weighted l2 norm, the 3D form of the 2D reading.
Run: python tests/golden/make_e1_3d_oracle.py  (several minutes, single core).
"""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_1611_02967_gb300 import inputs  # noqa: E402

L = 3.2


def trilinear(c):
    """Coarse cell-centred field to the grid of half the spacing: each fine
    cell takes 3/4 of its parent and 1/4 of the parent's neighbour on its side,
    per axis (27/64, 9/64, 3/64, 1/64 in total); ghosts mirror the boundary
    cell (Neumann)."""
    n = c.shape[0]
    g = np.pad(c, 1, mode="edge")
    f = np.empty((2 * n, 2 * n, 2 * n))
    for dk in (0, 1):
        for dj in (0, 1):
            for di in (0, 1):
                o = [-1 if d == 0 else 1 for d in (dk, dj, di)]
                acc = np.zeros((n, n, n))
                for sk in (0, 1):
                    for sj in (0, 1):
                        for si in (0, 1):
                            w = (3 if sk == 0 else 1) * (3 if sj == 0 else 1) * (3 if si == 0 else 1) / 64.0
                            a, b, e = 1 + sk * o[0], 1 + sj * o[1], 1 + si * o[2]
                            acc += w * g[a:a + n, b:b + n, e:e + n]
                f[dk::2, dj::2, di::2] = acc
    return f


def main():
    sol, nv = {}, {}
    for n in (8, 16, 32, 64):
        h = L / n
        s = 0.05 * h
        prm = oracle.Params(h, 0.2, 2.0, s, tol=1e-10)
        phi, _, _, _, counts = oracle.run(inputs.cosine_bump3(n, L), prm, int(round(0.8 / s)))
        sol[n], nv[n] = phi, float(np.mean(counts))
        print(n, nv[n], flush=True)
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "e1_3d_oracle.txt")
    with open(out, "w") as f:
        f.write("# CPU oracle, 3D version of the Table 1 setting (Section 5.1), written by make_e1_3d_oracle.py\n")
        f.write("# h_f denominator, ||delta phi||_2 (trilinear, h_f^3-weighted), mean V-cycles per step on h_f\n")
        for n in (16, 32, 64):
            d = sol[n] - trilinear(sol[n // 2])
            f.write("%d %.10e %.4f\n" % (n, np.sqrt((L / n) ** 3 * np.sum(d * d)), nv[n]))
    print(open(out).read())


if __name__ == "__main__":
    main()
