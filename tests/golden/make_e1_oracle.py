"""Write tests/golden/e1_oracle.txt: the CPU oracle's Cauchy differences for
the Table 1 setting of Section 5.1 (Eq. 5.1 on (0,3.2)^2, eps 0.2, gamma 2,
s = 0.05 h, T = 0.8, tol 1e-10), fine grids 32, 64, 128 and 256.

Calls only oracle/ (and the seedless Eq. 5.1 generator).  The Cauchy
difference uses cell-centred bilinear interpolation with mirrored ghosts and
the h_f-weighted l2 norm: Section 5.1 names bilinear interpolation and then
matlab's "nearest", but nearest injection between cell-centred grids is first
order and could not give the printed rates of 2, so bilinear is taken.
Run: python tests/golden/make_e1_oracle.py  (a few minutes, single core).
"""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_1611_02967_gb300 import inputs  # noqa: E402

L = 3.2


def bilinear(c):
    g = np.pad(c, 1, mode="edge")
    n = c.shape[0]
    f = np.empty((2 * n, 2 * n))
    for dj in (0, 1):
        for di in (0, 1):
            oj = -1 if dj == 0 else 1
            oi = -1 if di == 0 else 1
            C = g[1:-1, 1:-1]
            X = g[1:-1, 1 + oi:n + 1 + oi]
            Y = g[1 + oj:n + 1 + oj, 1:-1]
            D = g[1 + oj:n + 1 + oj, 1 + oi:n + 1 + oi]
            f[dj::2, di::2] = (9 * C + 3 * X + 3 * Y + D) / 16
    return f


def main():
    sol, nv = {}, {}
    for n in (16, 32, 64, 128, 256):
        h = L / n
        s = 0.05 * h
        prm = oracle.Params(h, 0.2, 2.0, s, tol=1e-10)
        phi, _, _, _, counts = oracle.run(inputs.cosine_bump(n, L), prm, int(round(0.8 / s)))
        sol[n], nv[n] = phi, float(np.mean(counts))
        print(n, nv[n], flush=True)
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "e1_oracle.txt")
    with open(out, "w") as f:
        f.write("# CPU oracle, Table 1 setting (Section 5.1), written by make_e1_oracle.py\n")
        f.write("# h_f denominator, ||delta phi||_2 (bilinear, h_f-weighted), mean V-cycles per step on h_f\n")
        for n in (32, 64, 128, 256):
            d = sol[n] - bilinear(sol[n // 2])
            f.write("%d %.10e %.4f\n" % (n, np.sqrt((L / n) ** 2 * np.sum(d * d)), nv[n]))
    print(open(out).read())


if __name__ == "__main__":
    main()
