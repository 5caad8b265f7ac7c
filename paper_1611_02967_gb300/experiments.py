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

The serving workload (not from the paper: a stream of runs of mixed
dimension, size and parameters served by the request loop):

    python -m paper_1611_02967_gb300.experiments OUT_PREFIX --study serving [--runs N]

writes OUT_PREFIX_runs.csv (one row per run: arrival, wait for admission,
latency, V-cycles) with the capacity and latency percentiles in its header.
"""
import argparse
import csv
import json

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


# ---------------------------------------------------------------- batched

def batched_runs(seed=4, nruns=256):
    """The batched workload's runs: sizes drawn from {64..1024}^2, eps
    U(0.02,0.08), gamma U(0.5,4), h 0.025, dt 0.005, seeded spinodal data.
    Returns (run descriptions (shape, h, eps, gamma, dt), initial fields,
    sizes)."""
    u = inputs.uniform01(seed, nruns * 3, stream=13).reshape(nruns, 3)
    sizes = np.array([64, 128, 256, 512, 1024])[np.minimum((u[:, 0] * 5).astype(int), 4)]
    runs = [((int(n), int(n)), 0.025, 0.02 + 0.06 * u[k, 1], 0.5 + 3.5 * u[k, 2], 0.005) for k, n in enumerate(sizes)]
    phis = [inputs.spinodal((int(n), int(n)), seed * 1000 + k, mean=0.0) for k, n in enumerate(sizes)]
    return runs, phis, sizes


# ---------------------------------------------------------------- serving

SERVE_SEED = 5
SERVE_POOL_BYTES = 48 << 30
SERVE_SLOTS = 12
SERVE_SLICE = 5


def serving_runs(nruns, seed=SERVE_SEED, steps=(10, 500)):
    """The serving workload's stream of runs, drawn from a seeded generator:
    half 2D (n in {128, 256, 512, 1024, 2048}^2, h 0.025, seeded spinodal
    noise about 0) and half 3D (n in {64, 128, 256}^3, h 0.05, four tanh
    bubbles up to 128^3, spinodal noise at 256^3), eps U(0.02, 0.08), gamma
    U(0.5, 4), dt 0.005, steps uniform in the given range.  Returns a list of
    dicts (shape, h, eps, gamma, steps, cells, phi0) and the uniform draws
    u_gap that set the arrival gaps (serve_arrivals)."""
    u = inputs.uniform01(seed, nruns * 7, stream=11).reshape(nruns, 7)
    three_d = u[:, 5] < 0.5
    n2 = np.array([128, 256, 512, 1024, 2048])[np.minimum((u[:, 0] * 5).astype(int), 4)]
    n3 = np.array([64, 128, 256])[np.minimum((u[:, 0] * 3).astype(int), 2)]
    sizes = np.where(three_d, n3, n2)
    nsteps = steps[0] + (u[:, 1] * (steps[1] - steps[0] + 1)).astype(int)
    eps = 0.02 + 0.06 * u[:, 2]
    gamma = 0.5 + 3.5 * u[:, 3]
    runs = []
    for k in range(nruns):
        n = int(sizes[k])
        if three_d[k]:
            shape, h = (n, n, n), 0.05
            phi0 = (inputs.bubbles(n, n * h, eps[k], seed * 1000 + k, count=4) if n <= 128
                    else inputs.spinodal(shape, seed * 1000 + k, mean=0.0))
        else:
            shape, h = (n, n), 0.025
            phi0 = inputs.spinodal(shape, seed * 1000 + k, mean=0.0)
        runs.append(dict(shape=shape, h=h, eps=float(eps[k]), gamma=float(gamma[k]), steps=int(nsteps[k]),
                         cells=int(np.prod(shape)), phi0=phi0))
    return runs, u[:, 4]


def serve_arrivals(runs, u_gap, rate_cell_steps_per_s):
    """Poisson arrival times (seconds from the first) whose offered work is
    rate_cell_steps_per_s on average: exponential gaps of mean
    (mean work per run) / rate."""
    work = np.array([r["cells"] * r["steps"] for r in runs], dtype=float)
    runs_per_s = rate_cell_steps_per_s / work.mean()
    return np.cumsum(-np.log(1.0 - u_gap) / runs_per_s)


def serve(runs, arrivals, dt=0.005, precision=1, pool_bytes=SERVE_POOL_BYTES, max_active=SERVE_SLOTS,
          steps_per_slice=SERVE_SLICE, timeout=3600.0):
    """Submit every run to one request loop (chhs_server_*) at its arrival
    time and wait for all.  Returns (per-run results, span in seconds from the
    first submission to the last completion)."""
    import time
    with chhs.Server(pool_bytes=pool_bytes, max_active=max_active, steps_per_slice=steps_per_slice) as sv:
        t0 = time.perf_counter()
        ids = []
        for r, t in zip(runs, arrivals):
            while time.perf_counter() < t0 + t:
                time.sleep(0.0002)
            ids.append(sv.submit(r["shape"], r["h"], r["eps"], r["gamma"], dt, r["steps"], r["phi0"],
                                 precision=precision))
        res = []
        for rid in ids:
            sv.wait(rid, timeout)
            res.append(sv.result(rid, with_phi=False))
            sv.release(rid)
    span = max(x["t_done"] for x in res) - min(x["t_submit"] for x in res)
    return res, span


def serving_summary(runs, res, span, load):
    work = np.array([r["cells"] * r["steps"] for r in runs], dtype=float)
    lat = np.array([x["t_done"] - x["t_submit"] for x in res])
    return dict(runs=len(runs), offered_load=load, p50_s=float(np.percentile(lat, 50)),
                p99_s=float(np.percentile(lat, 99)), mean_s=float(lat.mean()), max_s=float(lat.max()),
                value=float(work.sum() / span), span_s=float(span),
                all_converged=all(x["status"] == 0 for x in res),
                vcycles_per_step=float(sum(x["vcycles"] for x in res) / sum(r["steps"] for r in runs)))


def serving_study(nruns=100, load=0.8, seed=SERVE_SEED):
    """The serving workload with its full 10-500 step range: the capacity of
    the request loop measured on the stream itself (every run submitted at
    once, throughput = work / span), then the same runs as Poisson arrivals
    at `load` times that capacity; returns (summary, per-run rows)."""
    runs, u_gap = serving_runs(nruns, seed)
    closed, span_c = serve(runs, np.zeros(nruns))
    capacity = float(sum(r["cells"] * r["steps"] for r in runs) / span_c)
    res, span = serve(runs, serve_arrivals(runs, u_gap, load * capacity))
    summary = serving_summary(runs, res, span, load)
    summary["capacity"] = capacity
    summary["closed_p50_s"] = float(np.percentile([x["t_done"] - x["t_submit"] for x in closed], 50))
    rows = [dict(run=k, dim=len(r["shape"]), n=r["shape"][0], steps=r["steps"], eps=r["eps"], gamma=r["gamma"],
                 t_submit=x["t_submit"] - res[0]["t_submit"], wait_s=x["t_admit"] - x["t_submit"],
                 latency_s=x["t_done"] - x["t_submit"], vcycles=x["vcycles"], status=x["status"])
            for k, (r, x) in enumerate(zip(runs, res))]
    return summary, rows


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
    ap.add_argument("--study", choices=["gamma", "serving"], default="gamma")
    ap.add_argument("--runs", type=int, default=100, help="serving study: runs in the stream")
    args = ap.parse_args(argv)
    if args.study == "serving":
        summary, rows = serving_study(args.runs)
        head = ["serving workload, %d runs with 10-500 steps (SplitMix64 seed %d): half 2D n in {128..2048}^2, "
                "half 3D n in {64,128,256}^3, eps U(0.02,0.08), gamma U(0.5,4), dt 0.005, mixed precision; "
                "request loop with a %d GiB pool, %d slots, %d steps per slice" %
                (args.runs, SERVE_SEED, SERVE_POOL_BYTES >> 30, SERVE_SLOTS, SERVE_SLICE),
                "capacity (all runs submitted at once) %.4g cell-steps/s; Poisson arrivals at %.2f of it" %
                (summary["capacity"], summary["offered_load"]),
                "summary: " + json.dumps(summary),
                "written by: python -m paper_1611_02967_gb300.experiments %s --study serving --runs %d" %
                (args.prefix, args.runs)]
        write_csv(args.prefix + "_runs.csv", rows, head)
        print(json.dumps(summary))
        return
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
