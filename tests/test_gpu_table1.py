"""Table 1 of Section 5.1 reproduced on the GPU (double-precision form).

Eq. 5.1 on (0,3.2)^2, eps = 0.2, gamma = 2, s = 0.05 h, T = 0.8, FAS V(2,2)
to 1e-10, fine grids 3.2/32 ... 3.2/512 (160 ... 2560 steps).  The GPU's
Cauchy differences must equal the CPU oracle's (tests/golden/e1_oracle.txt,
written by make_e1_oracle.py from oracle/ only) for the grids the oracle can
afford, and the rates must be within 0.1 of the printed ones.  The printed
error magnitudes themselves are not matched by either side: both give
differences a steady factor of about 5 above the printed ones, and none of
the readings tried on the oracle (norm normalisation, nearest or bilinear
transfer, restriction-based comparison, start-up from a near-exact phi^1,
other T, s or gamma) lands within two digits of them.
"""
import os

import numpy as np
import pytest

from paper_1611_02967_gb300 import chhs, inputs

pytestmark = pytest.mark.gpu

L = 3.2
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _read(name):
    rows = []
    for line in open(os.path.join(GOLDEN, name)):
        line = line.split("#")[0].strip()
        if line and not line.startswith("mass0"):
            rows.append(line.split())
    return rows


def _bilinear(c):
    g = np.pad(c, 1, mode="edge")
    n = c.shape[0]
    f = np.empty((2 * n, 2 * n))
    for dj in (0, 1):
        for di in (0, 1):
            oj = -1 if dj == 0 else 1
            oi = -1 if di == 0 else 1
            f[dj::2, di::2] = (9 * g[1:-1, 1:-1] + 3 * g[1:-1, 1 + oi:n + 1 + oi]
                               + 3 * g[1 + oj:n + 1 + oj, 1:-1] + g[1 + oj:n + 1 + oj, 1 + oi:n + 1 + oi]) / 16
    return f


def test_table1_cauchy_convergence_on_gpu():
    sols, nv = {}, {}
    for n in (16, 32, 64, 128, 256, 512):
        h = L / n
        s = 0.05 * h
        steps = int(round(0.8 / s))
        with chhs.Run((n, n), h, 0.2, 2.0, s) as run:
            run.set_phi(inputs.cosine_bump(n, L))
            assert abs(run.mass() - (-5.12)) < 1e-12  # printed initial mass
            _, v, r = run.step(steps)
            assert r <= 1e-10
            assert abs(run.mass() - (-5.12)) < steps * 10.24 * 1.1e-10
            sols[n], nv[n] = run.get_phi(), v / steps
    err = {n: np.sqrt((L / n) ** 2 * np.sum((sols[n] - _bilinear(sols[n // 2])) ** 2)) for n in (32, 64, 128, 256, 512)}
    print("GPU Table 1:", {n: "%.4e (V %.2f)" % (err[n], nv[n]) for n in err})
    for n_s, e_s, v_s in _read("e1_oracle.txt"):
        n = int(n_s)
        assert abs(err[n] - float(e_s)) <= 1e-4 * float(e_s), (n, err[n], e_s)
    printed = {int(r[1]): (float(r[3]), int(r[4])) for r in _read("table1_cauchy.txt")}
    for n in (64, 128, 256, 512):
        rate = np.log2(err[n // 2] / err[n])
        assert abs(rate - printed[n][0]) <= 0.1, (n, rate, printed[n])
    for n in (32, 64, 128, 256, 512):
        assert abs(nv[n] - printed[n][1]) <= 1.5, (n, nv[n], printed[n])


def _golden_module(name):
    import importlib.util
    spec = importlib.util.spec_from_file_location(name, os.path.join(GOLDEN, name + ".py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_3d_cauchy_convergence_on_gpu():
    """A 3D version of the Table 1 experiment (the paper prints 2D only): the
    3D analogue of Eq. 5.1 on (0,3.2)^3 with the Table 1 parameters, grids 8^3
    ... 128^3.  The GPU's Cauchy differences equal the CPU oracle's
    (tests/golden/e1_3d_oracle.txt) where the oracle can afford them, the
    rates rise towards the scheme's second order, and mass is conserved
    (initial mass -3/4 L^3 in closed form)."""
    tri = _golden_module("make_e1_3d_oracle").trilinear
    sols, nv = {}, {}
    mass0 = -0.75 * L ** 3
    for n in (8, 16, 32, 64, 128):
        h = L / n
        s = 0.05 * h
        steps = int(round(0.8 / s))
        with chhs.Run((n, n, n), h, 0.2, 2.0, s) as run:
            run.set_phi(inputs.cosine_bump3(n, L))
            assert abs(run.mass() - mass0) < 1e-11
            _, v, r = run.step(steps)
            assert r <= 1e-10
            assert abs(run.mass() - mass0) < steps * L ** 3 * 1.1e-10
            sols[n], nv[n] = run.get_phi(), v / steps
    err = {n: np.sqrt((L / n) ** 3 * np.sum((sols[n] - tri(sols[n // 2])) ** 2)) for n in (16, 32, 64, 128)}
    rate = {n: np.log2(err[n // 2] / err[n]) for n in (32, 64, 128)}
    print("GPU 3D Cauchy:", {n: "%.4e (V %.2f)" % (err[n], nv[n]) for n in err}, "rates", rate)
    for n_s, e_s, v_s in _read("e1_3d_oracle.txt"):
        n = int(n_s)
        assert abs(err[n] - float(e_s)) <= 1e-4 * float(e_s), (n, err[n], e_s)
    assert rate[32] < rate[64] < rate[128] + 0.05
    assert abs(rate[128] - 2.0) <= 0.2, rate
