"""Write tests/golden/dt_sweep512_oracle.txt: the CPU oracle's Cauchy
differences under time-step halving on the 512 x 512 grid of the 2D
spinodal configuration ((0,12.8)^2, h = 0.025, eps 0.05, gamma 1), from the
smooth initial field of Eq. 5.1 scaled to L = 12.8, to T = 0.2 with
s = 0.02, 0.01, 0.005, 0.0025, 0.00125 (10 ... 160 steps), tol 1e-12.

The main convergence theorem gives O(s^2 + h^2); at fixed h the Cauchy
differences ||phi_s - phi_{s/2}||_2 (h-weighted l2) fall by a factor that
tends to 4 as s shrinks.  (The seeded random field of the configuration
itself is too rough for the ratios to settle at these s.)
Calls only oracle/ and the seedless Eq. 5.1 generator.
Run: python tests/golden/make_dt_sweep512.py  (a few minutes on 5 cores).
"""
import multiprocessing as mp
import os
import sys
from concurrent.futures import ProcessPoolExecutor

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_1611_02967_gb300 import inputs  # noqa: E402

N, L, EPS, GAMMA, T, TOL = 512, 12.8, 0.05, 1.0, 0.2, 1e-12
DTS = (0.02, 0.01, 0.005, 0.0025, 0.00125)


def solve(s):
    h = L / N
    return oracle.run(inputs.cosine_bump(N, L), oracle.Params(h, EPS, GAMMA, s, tol=TOL), int(round(T / s)))[0]


def main():
    with ProcessPoolExecutor(len(DTS), mp_context=mp.get_context("spawn")) as ex:
        sols = dict(zip(DTS, ex.map(solve, DTS)))
    h = L / N
    diffs = [float(np.sqrt(h * h * np.sum((sols[DTS[k]] - sols[DTS[k + 1]]) ** 2))) for k in range(len(DTS) - 1)]
    with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "dt_sweep512_oracle.txt"), "w") as f:
        f.write("# Cauchy differences under dt halving, 512^2, Eq. 5.1 scaled to L = 12.8, eps 0.05, gamma 1,\n")
        f.write("# T = 0.2, tol 1e-12; written by tests/golden/make_dt_sweep512.py (oracle/ only)\n")
        f.write("# columns: s, s/2, ||phi_s - phi_{s/2}||_2\n")
        for k in range(len(DTS) - 1):
            f.write("%.6g %.6g %.10e\n" % (DTS[k], DTS[k + 1], diffs[k]))


if __name__ == "__main__":
    main()
