"""The spinodal-decomposition study of Section 5.2, run through the C ABI.

512 x 512 cells on (0, 6.4)^2 (h = 6.4/512), eps = 0.03, s = 0.01,
phi0 = -0.05 + 0.05 (2 r - 1) with r uniform per cell, gamma in {0, 2, 4},
to t = 5 (500 steps).  Every step records the discrete energy E_h
(Eq. 2.8), the modified energy F_h (Eq. 2.9), the mass, the dissipation
terms s ||grad_h mu||^2 and (s/gamma) ||u||^2 of Eq. 2.23 and the V-cycles;
at the paper's snapshot times (t = 0.5, 1, 3, 5) it records a few
statistics of the phase field: the particles (connected sets of cells with
phi > 0), their mean area and mean shape factor P^2 / (4 pi A) (perimeter P
counted over the cell faces between the phases; 1 for a disc, larger for
elongated particles).

    python -m paper_1611_02967_gb300.experiments OUT_PREFIX [--precision 0|1]

writes OUT_PREFIX_energy.csv (one row per step and gamma) and
OUT_PREFIX_snapshots.csv.  The paper plots these curves and snapshots
(Figs. 2-3) but prints no values.
"""
import argparse
import csv

import numpy as np

from . import chhs, inputs

L_DOMAIN, N, EPS, DT, STEPS = 6.4, 512, 0.03, 0.01, 500
SNAPSHOT_STEPS = (50, 100, 300, 500)  # t = 0.5, 1, 3, 5
SEED = 52


def initial_field():
    return inputs.spinodal((N, N), SEED, mean=-0.05, amplitude=0.05)


def particle_stats(phi, h):
    """Particles of {phi > 0} (4-connected), their mean area and mean shape
    factor P^2 / (4 pi A)."""
    from scipy import ndimage
    inside = phi > 0.0
    labels, count = ndimage.label(inside)
    if count == 0:
        return dict(particles=0, mean_area=0.0, mean_shape_factor=0.0, phase_fraction=0.0)
    area = np.bincount(labels.ravel(), minlength=count + 1)[1:] * h * h
    per = np.zeros(count + 1)
    # faces between a particle cell and a cell outside it (the domain
    # boundary does not count: homogeneous Neumann walls are not interfaces)
    for a, b in ((labels[:, :-1], labels[:, 1:]), (labels[:-1, :], labels[1:, :])):
        diff = a != b
        np.add.at(per, a[diff], h)
        np.add.at(per, b[diff], h)
    per = per[1:]
    shape = per * per / (4.0 * np.pi * area)
    return dict(particles=int(count), mean_area=float(area.mean()), mean_shape_factor=float(shape.mean()),
                phase_fraction=float(inside.mean()))


def gamma_study(gammas=(0.0, 2.0, 4.0), steps=STEPS, precision=0, sample_steps=(), on_sample=None):
    """Run the study.  For each step k in sample_steps, on_sample(gamma, k,
    before, phi) receives the state (phi^m, phi^{m-1}, mu, p) that step k
    started from and the phi it produced.  Returns (rows, snapshots)."""
    h = L_DOMAIN / N
    rows, snaps = [], []
    for gamma in gammas:
        with chhs.Run((N, N), h, EPS, gamma, DT, opts=chhs.default_opts(precision=precision)) as run:
            run.set_phi(initial_field())
            E, F = run.energy()
            rows.append(dict(gamma=gamma, step=0, t=0.0, E=E, F=F, mass=run.mass(), diss_mu=0.0, diss_u=0.0,
                             u_sq=0.0, vcycles=0))
            for k in range(1, steps + 1):
                before = run.get_state() if k in sample_steps else None
                _, v, _ = run.step(1)
                E, F = run.energy()
                gmu, u2, _ = run.dissipation()
                rows.append(dict(gamma=gamma, step=k, t=k * DT, E=E, F=F, mass=run.mass(), diss_mu=DT * gmu,
                                 diss_u=(DT / gamma * u2) if gamma > 0 else 0.0, u_sq=u2, vcycles=v))
                if before is not None and on_sample is not None:
                    on_sample(gamma, k, before, run.get_phi())
                if k in SNAPSHOT_STEPS:
                    snaps.append(dict(gamma=gamma, step=k, t=k * DT, **particle_stats(run.get_phi(), h)))
    return rows, snaps


def write_csv(path, rows, header):
    with open(path, "w", newline="") as f:
        for line in header:
            f.write("# " + line + "\n")
        w = csv.DictWriter(f, fieldnames=list(rows[0].keys()))
        w.writeheader()
        for r in rows:
            w.writerow({k: (repr(v) if isinstance(v, float) else v) for k, v in r.items()})


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("prefix")
    ap.add_argument("--precision", type=int, default=0)
    args = ap.parse_args(argv)
    rows, snaps = gamma_study(precision=args.precision)
    head = ["Section 5.2 spinodal study: 512^2 on (0,6.4)^2, eps 0.03, s 0.01, phi0 = -0.05 + 0.05(2r-1) "
            "(SplitMix64 seed %d), gamma in {0,2,4}, t = 0..5; %s form, residual 1e-10" %
            (SEED, "double-precision" if args.precision == 0 else "mixed-precision"),
            "written by: python -m paper_1611_02967_gb300.experiments %s --precision %d" % (args.prefix,
                                                                                            args.precision)]
    write_csv(args.prefix + "_energy.csv", rows, head + ["E = E_h (Eq. 2.8), F = F_h (Eq. 2.9), "
                                                         "diss_mu = s||grad mu||^2, diss_u = (s/gamma)||u||^2, u_sq = ||u||^2"])
    write_csv(args.prefix + "_snapshots.csv", snaps,
              head + ["particles: 4-connected sets of cells with phi > 0; shape factor P^2/(4 pi A)"])


if __name__ == "__main__":
    main()
