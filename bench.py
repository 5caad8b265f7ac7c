#!/usr/bin/env python
"""Benchmark: CHHS cell-steps/s of the per-step FAS solve at residual 1e-10.

A benchmark step is one time step of the 512 x 512 spinodal workload (2D,
(0,12.8)^2, eps 0.05, gamma 1, dt 0.005, seeded noise of amplitude 0.05
about mean 0): one full FAS solve of Eqs. 2.5-2.7 to the 1e-10 stopping norm,
run through the C ABI.  A cell-step is one cell advanced one time step.
Before each timed region the handle's launch shapes are picked by
chhs_autotune on its own problem (untimed, like the warm-up; the state is
restored) and reported under "tuning".

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

One process per GPU (torchrun for N > 1); every rank runs its own replica of
the workload (runs are independent, so the path shards only across runs),
the time is the maximum over ranks and `value` counts the cell-steps of all
ranks.  Rank 0 prints one JSON line.

`--impl reference` times the CPU oracle (the plain double-precision
lexicographic FAS of ``oracle/``) on the host cores instead, on rank 0 only.
"""
import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "CHHS cell-steps/s at 1e-10 residual, mixed vs FP64 form; served p50/p99"
UNIT = "cell-steps/s"
WORKLOAD = "spinodal512"
WORKLOAD_DESC = ("2D spinodal 512x512 on (0,12.8)^2, Neumann, eps=0.05, gamma=1, dt=0.005, "
                 "phi0 = 0.05*U(-1,1) (SplitMix64 seed 2), FAS V(2,2) to residual 1e-10, FP64")
L2_FLUSH_BYTES = 256 << 20
# Nominal FP64 peak of a GB300: 152 SMs x 2070 MHz x 4 FP64 flop/clk/SM
# (2 DFMA per clock per SM) = 1.2586 TFLOP/s.
FP64_PEAK_TFLOPS = 152 * 2.070e9 * 4 / 1e12
# Algorithmic FP64 flops of one smoother cell update (interior cell with n
# faces), counted from the formulas k_smooth evaluates (add/sub/mul = 1,
# fma = 2, the reciprocal = 1).  Neighbour sums: sum (M mu_e + a p_e) 4n - 1,
# sum a mu_e 2n - 1, sum phi_e and sum p_e n - 1 each: 8n - 4.  Per cell: R1 (7),
# R2 with the cubic (9), B (4), R3 / Dn (9), dphi with 1 + Ae B and its
# reciprocal (8), dmu (2), dp (2), the three updates (3) = 44 (phi^m / 4 is a
# stored per-step constant).
SMOOTH_FLOPS = {2: 8 * 4 - 4 + 44, 3: 8 * 6 - 4 + 44}
# The byte model of one smoothing pass per cell (both colours, in order): read
# phi, mu, p, phi^m, phi*, f_mu and write phi, mu, p, nine values; per colour
# launch half of it per cell of the level.  In double precision 72 B per cell
# updated; in the single-precision correction form the pass reads the
# correction (3), the right-hand sides (3), phi^m, phi* and phi_b and writes
# the correction, twelve 4-byte values: 24 B per cell of the level per colour
# launch.
SMOOTH_BYTES_F64 = 72.0
SMOOTH_BYTES_F32_PER_CELL_PER_COLOUR = 24.0


L2_PROBE_SOURCE = ("measured: chhs_probe_l2 (48 MiB held in the L2, read 50 times by every SM with L1-bypassing "
                   "16-byte loads, best of 3) in this run")


def l2_peak():
    """Measured L2 read bandwidth (GB/s) of this GPU, best of three probes
    (None if the probe fails: the L2 figures are then left out)."""
    from paper_1611_02967_gb300 import chhs
    try:
        return max(chhs.probe_l2() for _ in range(3))
    except chhs.ChhsError:
        return None


def l2_roofline(alg_bytes, secs, peak, lts_bytes, why):
    """The kernel against the L2's read bandwidth: its algorithmic bytes, and
    the L1<->L2 request bytes ncu counted for it (l1tex__m_xbar2l1tex_read_bytes
    + l1tex__m_l1tex2xbar_write_bytes, when the summary matches the source;
    the quantity the probe measures), per launch over its duration."""
    if not peak:
        return {"peak_gbs": None, "note": "the L2 probe failed"}
    out = {"peak_gbs": peak, "peak_source": L2_PROBE_SOURCE, "algorithmic_gbs": alg_bytes / secs / 1e9,
           "frac_algorithmic": alg_bytes / secs / 1e9 / peak, "traffic": lts_bytes, "note": why}
    if lts_bytes:
        out["achieved_gbs"] = lts_bytes / secs / 1e9
        out["frac"] = lts_bytes / secs / 1e9 / peak
    return out


def hbm_peak():
    """(GB/s, source): the measured copy bandwidth of this GPU pool written
    beside the repository, else the recipe's fallback figure."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured (copy bandwidth of this pool's GB300s)"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback (6.8 TB/s, one earlier GB300 measurement)"
KERNEL_SRC = os.path.join(ROOT, "paper_1611_02967_gb300", "csrc", "chhs_kernels.cuh")
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "k_smooth_spinodal512.txt")
KERNEL_SRC_3D = os.path.join(ROOT, "paper_1611_02967_gb300", "csrc", "chhs_corr3.cuh")
TRAFFIC_FILE_3D = os.path.join(ROOT, "profiles", "k_smooth_c_bubbles128.txt")
TRAFFIC_FILE_256 = os.path.join(ROOT, "profiles", "k_smooth_c4_bubbles256.txt")


def parse_args(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true", help="skip the oracle timing leg")
    ap.add_argument("--no-request-loop", action="store_true",
                    help="skip the served and batched legs (for profiler runs: their request loops "
                         "launch for minutes under a profiler)")
    ap.add_argument("--profile-run", choices=PROFILE_RUNS, default=None,
                    help="for profiler captures: only W graph steps of one workload and form, then K steps "
                         "launched kernel by kernel (chhs_profile_step, which a profiler can see), and a "
                         "JSON line of the per-kernel-kind device times")
    return ap.parse_args(argv)


PROFILE_RUNS = ["spinodal512-f64", "spinodal512-mixed", "bubbles128-f64", "bubbles128-mixed",
                "spinodal64-f64", "spinodal64-mixed", "bubbles256-mixed", "batched-mixed"]


def profile_run(args):
    """W steps through the step graph, then K steps launched kernel by kernel
    with CUDA events (the form profilers can capture: they do not see inside
    a graph with a conditional node); prints the per-kind times."""
    import torch

    from paper_1611_02967_gb300 import chhs, inputs
    name, form = args.profile_run.rsplit("-", 1)
    if name == "batched":
        return profile_batched(args)
    w = inputs.workload(name)
    run = chhs.Run(w["shape"], w["h"], w["eps"], w["gamma"], w["dt"],
                   opts=chhs.default_opts(precision=1 if form == "mixed" else 0))
    run.set_phi(w["phi0"])
    if args.warmup:
        run.step(args.warmup)
    prof = None
    for _ in range(args.steps):
        prof = run.profile_step(prof)
    torch.cuda.synchronize()
    total = sum(v[0] for v in prof.values())
    print(json.dumps({"profile_run": args.profile_run, "steps": args.steps, "ms_per_step": total / args.steps,
                      "kernels": {k: {"ms_per_step": v[0] / args.steps, "share": v[0] / total,
                                      "launches_per_step": v[1] / args.steps,
                                      "us_per_launch": 1e3 * v[0] / v[1] if v[1] else None}
                                  for k, v in prof.items()}}), flush=True)
    run.close()
    return 0


def profile_batched(args):
    """The batched configuration (256 runs, mixed form, default tuning): W
    steps through the batch's graph, then K steps launched kernel by kernel
    (chhs_batch_profile_step); prints the per-kind times."""
    import torch

    from paper_1611_02967_gb300 import chhs
    runs, phis, sizes = batched_runs()
    with chhs.Batch(runs) as b:
        for k in range(len(runs)):
            b.runs[k].set_phi(phis[k])
        if args.warmup:
            b.step(args.warmup)
        prof = None
        for _ in range(args.steps):
            prof = b.profile_step(prof)
        torch.cuda.synchronize()
    total = sum(v[0] for v in prof.values())
    print(json.dumps({"profile_run": args.profile_run, "steps": args.steps, "ms_per_step": total / args.steps,
                      "kernels": {k: {"ms_per_step": v[0] / args.steps, "share": v[0] / total,
                                      "launches_per_step": v[1] / args.steps} for k, v in prof.items()}}),
          flush=True)
    return 0


def dist_env():
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def config(world):
    return {"workload": WORKLOAD_DESC, "cells": 512 * 512, "workload_steps": 200,
            "l2": "flushed between timed steps (256 MiB device write, untimed)",
            "parallelism": "replicas x%d (one independent run per GPU)" % world}


def kernel_hash():
    """Hash of the part of the kernel header that defines k_smooth and what it
    calls (everything before the transfer kernels), so that edits to other
    kernels do not invalidate the smoother's recorded traffic."""
    with open(KERNEL_SRC, "rb") as f:
        src = f.read()
    cut = src.find(b"// ---------------------------------------------------------------- transfers")
    return hashlib.sha256(src[:cut if cut > 0 else len(src)]).hexdigest()[:16]


def file_hash(path):
    """Hash of a kernel source file up to its restriction section (the 3D
    colour pass and what it calls; a recorded traffic figure holds while it
    matches)."""
    with open(path, "rb") as f:
        src = f.read()
    cut = src.find(b"// ---------------------------------------------------------------- restriction")
    return hashlib.sha256(src[:cut if cut > 0 else len(src)]).hexdigest()[:16]


def measured_traffic(path=None, src=None, key="dram_bytes_per_launch"):
    """DRAM bytes per launch (or another per-launch figure, key) of the
    profiled kernel from a committed ncu summary (default: the
    double-precision smoother's), if it was taken on the current kernel
    source; else None."""
    path = path or TRAFFIC_FILE
    try:
        vals = {}
        with open(path) as f:
            for line in f:
                if "=" in line and not line.startswith("#"):
                    k, v = line.split("=", 1)
                    vals[k.strip()] = v.strip()
        if vals.get("kernel_source_sha256_16") != (kernel_hash() if src is None else file_hash(src)):
            return None
        return float(vals[key])
    except (OSError, KeyError, ValueError):
        return None


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.rows = []
        self.proc = None
        self.gpu = gpu_index
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits", "-lms", "200",
                 "-i", str(self.gpu)], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()
        t0 = time.time()
        while not self.rows and time.time() - t0 < 5.0:
            time.sleep(0.05)

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        return self.summarize(self.rows)

    @staticmethod
    def summarize(rows):
        """Median SM clock, the maximum clock and the throttle reasons seen
        active in nvidia-smi rows of FIELDS (values split, no header)."""
        rows = [r for r in rows if len(r) >= 9]
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[q] for r in rows for q in range(4) if r[5 + q].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def cpu_info():
    """(model name, online cores) of the host."""
    model = None
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith(("model name", "cpu model")):
                    model = line.split(":", 1)[1].strip()
                    break
    except OSError:
        pass
    if model is None:  # Arm hosts list no model name in /proc/cpuinfo; lscpu does
        try:
            out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
            for line in out.splitlines():
                if line.strip().lower().startswith("model name"):
                    model = line.split(":", 1)[1].strip()
                    break
        except (OSError, subprocess.SubprocessError):
            pass
    if model is None:
        import platform
        model = platform.processor() or platform.machine()
    return model, os.cpu_count()


def oracle_rate(w, max_seconds=15.0, max_steps=40, skip_first=True):
    """The CPU oracle as it stands, single-threaded, on the first steps of the
    workload: returns (cell-steps/s, steps timed, seconds)."""
    import numpy as np

    import oracle
    prm = oracle.Params(w["h"], w["eps"], w["gamma"], w["dt"], tol=1e-10)
    phim = np.array(w["phi0"], dtype=np.float64)
    phimm1 = phim.copy()
    mu = np.zeros_like(phim)
    p = np.zeros_like(phim)
    n = phim.size
    timed, t_total, k = 0, 0.0, 0
    while k < max_steps:
        t0 = time.perf_counter()
        phi, mu, p, v, r, st = oracle.step(phim, phimm1, prm, 2.0 * phim - phimm1, mu, p)
        dt = time.perf_counter() - t0
        if st != oracle.OK:
            raise RuntimeError("oracle step failed: %d" % st)
        phimm1, phim = phim, phi
        if k > 0 or not skip_first:
            timed += 1
            t_total += dt
        k += 1
        if t_total >= max_seconds:
            break
    return n * timed / t_total, timed, t_total


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    from paper_1611_02967_gb300 import inputs
    w = inputs.workload(WORKLOAD)
    n = 512 * 512
    import numpy as np

    import oracle
    prm = oracle.Params(w["h"], w["eps"], w["gamma"], w["dt"], tol=1e-10)
    phim = np.array(w["phi0"])
    phimm1 = phim.copy()
    mu = np.zeros_like(phim)
    p = np.zeros_like(phim)
    times, vs = [], []
    for k in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        phi, mu, p, v, r, st = oracle.step(phim, phimm1, prm, 2.0 * phim - phimm1, mu, p)
        t = time.perf_counter() - t0
        if st != oracle.OK:
            raise RuntimeError("oracle step %d failed: %d" % (k, st))
        phimm1, phim = phim, phi
        if k >= args.warmup:
            times.append(t)
            vs.append(v)
    total = sum(times)
    value = n * len(times) / total
    sample = "time steps %d..%d of the 512x512 workload, one oracle process" % (
        args.warmup + 1, args.warmup + args.steps)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / len(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": dict(config(1), l2="not applicable (host CPU)"),
            "vcycles_per_step": sum(vs) / len(vs),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample,
                             "cpu_model": cpu_info()[0], "nproc": cpu_info()[1]},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def reduce_max(value, world):
    """Max of a float over ranks (identity for one rank)."""
    if world == 1:
        return value
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([value], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def reduce_sum(value, world):
    if world == 1:
        return value
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([value], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def time_steps(run, steps, stream, flush):
    """K steps, each preceded by an untimed L2 flush and bracketed by CUDA
    events on the solver's stream.  All K are enqueued before the one wait, so
    the host's launch work overlaps the device's and the events see device
    time only.  Returns (device ms, V-cycles, last norm)."""
    import torch
    ev0 = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    ev1 = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    for k in range(steps):
        with torch.cuda.stream(stream):
            flush.fill_(k & 0xFF)
        ev0[k].record(stream)
        run.step_async(1)
        ev1[k].record(stream)
    _, vtot, resid = run.wait()
    torch.cuda.synchronize()
    return sum(a.elapsed_time(b) for a, b in zip(ev0, ev1)), vtot, resid


SERVED_DESC = ("served sample of the serving configuration: 60 runs, half 2D (n in {128, 256, 512, 1024, "
               "2048}^2, h 0.025, seeded spinodal) and half 3D (n in {64, 128, 256}^3, h 0.05, 4 tanh bubbles "
               "up to 128^3, seeded spinodal at 256^3), 10-50 steps (the configuration's 10-500 shortened so the "
               "sample ends in about half a minute), eps U(0.02,0.08), gamma U(0.5,4), dt 0.005, mixed precision, "
               "Poisson arrivals at about 0.8 of the measured mixed-form capacity, seed 5; 48 GiB pool, 12 "
               "active slots, 5 steps per slice")


def served_leg(capacity_cell_steps_per_s, nruns=60):
    """Continuous batching through chhs_server_*: latency percentiles and
    throughput of a seeded Poisson stream of runs drawn from the serving
    configuration's size and parameter ranges (experiments.serving_runs),
    with the step range shortened to 10-50 so that the leg ends in about
    half a minute."""
    from paper_1611_02967_gb300 import experiments as ex
    runs, u_gap = ex.serving_runs(nruns, steps=(10, 50))
    res, span = ex.serve(runs, ex.serve_arrivals(runs, u_gap, 0.8 * capacity_cell_steps_per_s))
    out = ex.serving_summary(runs, res, span, 0.8)
    out.update(unit=UNIT, sample=SERVED_DESC)
    return out


def e2e_steps(run, state, steps, ncell):
    """K steps through the public API with the state in pinned host memory:
    each step copies (phi^m, phi^{m-1}, mu, p) in, solves, and copies them
    out.  Returns (seconds, bytes in per step, bytes out per step)."""
    import torch

    from paper_1611_02967_gb300 import chhs
    host = [torch.empty(s_.shape, dtype=torch.float64, pin_memory=True).numpy() for s_ in state]
    for h_, s_ in zip(host, state):
        h_[...] = s_
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(steps):
        run.set_state(*host)
        run.step(1)
        chhs.lib().chhs_get_state(run.handle, *[chhs._buf(h_, ncell, True)[0] for h_ in host], 0)
    torch.cuda.synchronize()
    return time.perf_counter() - t0, 4 * 8 * ncell, 4 * 8 * ncell


def bubbles_leg(stream, flush, steps=10, warmup=3):
    """The 128^3 bubble workload (3D, eps 0.04, gamma 2, dt 0.005), the
    largest single-run configuration: both forms device-timed like the main
    line from the same state after warm-up, each with its end-to-end rate
    through the public API (host state copied in and out every step), and the
    HBM roofline of the mixed form's dominant memory-bound kernel, the
    finest-level single-precision colour pass."""
    from paper_1611_02967_gb300 import chhs, inputs
    w = inputs.workload("bubbles128")
    ncell = 128 ** 3
    out = {"workload": "3D bubbles 128^3 on (0,6.4)^3, eps 0.04, gamma 2, dt 0.005, 8 tanh bubbles (seed 3)",
           "steps": steps, "l2": "inputs larger than L2 (the 128^3 hierarchy is ~400 MB), and flushed between steps"}
    state = None
    for prec, key in ((0, "f64"), (1, "mixed")):
        run = chhs.Run(w["shape"], w["h"], w["eps"], w["gamma"], w["dt"], stream=stream.cuda_stream,
                       opts=chhs.default_opts(precision=prec))
        run.set_phi(w["phi0"])
        if state is None:
            run.step(warmup)
            state = run.get_state()
        run.set_state(*state)
        tune = run.autotune(2)
        run.set_state(*state)
        ms, v, r = time_steps(run, steps, stream, flush)
        secs, bi, bo = e2e_steps(run, state, steps, ncell)
        out[key] = {"value": ncell * steps / (ms / 1e3), "unit": UNIT, "ms_per_step": ms / steps,
                    "vcycles_per_step": v / steps, "final_resid": r, "tuning": tune,
                    "e2e": {"value": ncell * steps / secs, "unit": UNIT, "h2d_bytes_per_step": bi,
                            "d2h_bytes_per_step": bo}}
        if prec == 1:
            run.set_state(*state)
            run.step(1)
            t = run.profile_smooth32(100) / 1e3
            alg = SMOOTH_BYTES_F32_PER_CELL_PER_COLOUR * ncell
            gbs, src = hbm_peak()
            out[key]["roofline"] = {
                "bound": "hbm", "kernel": ("k_smooth_c4<0,0>" if tune.get("quad_passes", 1) else "k_smooth_c<3>")
                + " on the 128^3 level (single-precision colour pass, coefficients recomputed from phi*"
                + (", four cells of a row per thread)" if tune.get("quad_passes", 1) else ")"),
                "achieved": alg / t / 1e9, "peak": gbs, "unit": "GB/s", "frac": alg / t / 1e9 / gbs,
                "peak_source": src, "traffic": measured_traffic(TRAFFIC_FILE_3D, KERNEL_SRC_3D),
                "l2": l2_roofline(alg, t, l2_peak(), measured_traffic(TRAFFIC_FILE_3D, KERNEL_SRC_3D,
                                                                      "l2_request_bytes_per_launch"),
                                  "warm, the level's nine fields (75 MB) largely stay in the L2 between passes"),
                "algorithmic_bytes_per_launch": alg, "avg_launch_us": 1e6 * t,
                "duration_source": "100 launches back to back between CUDA events (chhs_profile_smooth32)",
                "note": "24 B per cell per colour launch: the twelve 4-byte values of a sweep (read correction, "
                        "right-hand sides, phi^m, phi*, phi_b; write the correction) split over its two launches",
                "grid_256": pass_256(stream)}
        run.close()
    return out


def pass_256(stream, npasses=50):
    """The same finest-level colour pass on the 256^3 bubbles grid (the
    largest 3D grid of the serving configuration, h 0.05), whose level fields
    (~600 MB) do not fit in the L2: back to back, against the byte model and
    the HBM peak."""
    from paper_1611_02967_gb300 import chhs, inputs
    w = inputs.workload("bubbles256")
    ncell = 256 ** 3
    run = chhs.Run(w["shape"], w["h"], w["eps"], w["gamma"], w["dt"], stream=stream.cuda_stream,
                   opts=chhs.default_opts(precision=1))
    try:
        run.set_phi(w["phi0"])
        run.step(1)
        t = run.profile_smooth32(npasses) / 1e3
    finally:
        run.close()
    alg = SMOOTH_BYTES_F32_PER_CELL_PER_COLOUR * ncell
    gbs, src = hbm_peak()
    traffic = measured_traffic(TRAFFIC_FILE_256, KERNEL_SRC_3D)
    out = {"workload": "3D bubbles 256^3 on (0,12.8)^3, eps 0.04, gamma 2, dt 0.005, 8 tanh bubbles (seed 3), "
                       "after one step", "achieved": alg / t / 1e9, "peak": gbs, "unit": "GB/s",
           "frac": alg / t / 1e9 / gbs, "peak_source": src, "algorithmic_bytes_per_launch": alg,
           "traffic": traffic, "avg_launch_us": 1e6 * t,
           "duration_source": "%d launches back to back between CUDA events (chhs_profile_smooth32)" % npasses}
    if traffic:  # the DRAM bytes ncu counted per launch, over the same duration
        out["traffic_gbs"] = traffic / t / 1e9
        out["traffic_frac"] = traffic / t / 1e9 / gbs
    return out


def batched_runs(seed=4, nruns=256):
    from paper_1611_02967_gb300 import experiments
    return experiments.batched_runs(seed, nruns)


def batched_leg(seed=4, nruns=256, steps=100, request_loop=True):
    """The batched workload in full (256 runs, 100 steps each, mixed
    precision) through chhs_batch: one graph of batched launches, one per
    kernel and multigrid level over all runs, its tail size and coarse sweep
    counts picked by chhs_batch_autotune, timed with CUDA events on the
    batch's stream (creation, tuning and initial data untimed).  For comparison the
    same runs also go through the request loop (32 runs on per-run streams)."""
    import numpy as np
    import torch

    from paper_1611_02967_gb300 import chhs
    runs, phis, sizes = batched_runs(seed, nruns)
    work = float((sizes.astype(float) ** 2).sum() * steps)
    stream = torch.cuda.Stream()
    with chhs.Batch(runs, stream=stream.cuda_stream) as b:
        for k in range(nruns):
            b.runs[k].set_phi(phis[k])
        tune = b.autotune(2)  # untimed; every run's state is restored
        per_v, per_step = b.launch_counts()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        st, v, r = b.step(steps)
        e1.record(stream)
        torch.cuda.synchronize()
        secs = e0.elapsed_time(e1) / 1e3
    out = {"value": work / secs, "unit": UNIT, "runs": nruns, "steps_each": steps, "seconds": secs,
           "all_converged": all(x == 0 for x in st), "vcycles_per_step": float(np.mean(v)) / steps,
           "launches_per_vcycle": per_v, "launches_per_step_frame": per_step, "tuning": tune,
           "sample": "%d runs (sizes drawn from {64..1024}^2, seed 4), %d steps each, one chhs_batch (mixed "
                     "precision)%s" % (nruns, steps, "; the full batched configuration" if (nruns, steps) == (256, 100)
                                       else "")}
    if request_loop:
        with chhs.Server(pool_bytes=16 << 30, max_active=32, steps_per_slice=5) as sv:
            ids = [sv.submit(sh, h, eps, gamma, dt, steps, phis[k], precision=1)
                   for k, (sh, h, eps, gamma, dt) in enumerate(runs)]
            for rid in ids:
                sv.wait(rid, 600.0)
            res = [sv.result(rid, with_phi=False) for rid in ids]
        span = max(x["t_done"] for x in res) - min(x["t_submit"] for x in res)
        out["request_loop"] = {"value": work / span, "unit": UNIT, "seconds": span,
                               "all_converged": all(x["status"] == 0 for x in res),
                               "sample": "the same runs submitted at t = 0 to the request loop (32 slots, per-run "
                                         "streams and graphs), wall clock from first submit to last result"}
    return out


def run_ours(args):
    import numpy as np
    import torch

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_1611_02967_gb300 import chhs, inputs
    w = inputs.workload(WORKLOAD)
    shape, ncell = w["shape"], 512 * 512
    stream = torch.cuda.Stream()
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device="cuda")
    run = chhs.Run(shape, w["h"], w["eps"], w["gamma"], w["dt"], stream=stream.cuda_stream)
    run.set_phi(w["phi0"])

    sampler = ClockSampler(torch.cuda.current_device()) if rank == 0 else None
    if sampler:
        sampler.start()
    # warm-up and launch-shape autotuning (both untimed; the tuner restores the state)
    run.step(args.warmup)
    tuning = {"f64": run.autotune(3)}
    per_v, per_step = run.launch_counts()
    state0 = run.get_state()  # the e2e leg below replays the same K steps
    # timed region: K steps, L2 flushed before each, device time by events
    barrier(world)
    torch.cuda.synchronize()
    dev_ms, vtot, resid = time_steps(run, args.steps, stream, flush)
    torch.cuda.synchronize()
    barrier(world)
    clocks = sampler.stop() if sampler else None
    max_ms = reduce_max(dev_ms, world)
    units = reduce_sum(float(ncell * args.steps), world)
    value = units / (max_ms / 1e3)
    checks = run.norm_checks()  # stopping norms after V-cycles: one kernel each
    launches = 1 + args.steps * per_step + vtot * per_v + checks

    # end to end through the public API with host-resident state: every step
    # copies (phi^m, phi^{m-1}, mu, p) in from pinned host memory, solves, and
    # copies them back out
    host = [torch.empty(shape, dtype=torch.float64, pin_memory=True).numpy() for _ in range(4)]
    for h_, s_ in zip(host, state0):
        h_[...] = s_
    barrier(world)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for k in range(args.steps):
        run.set_state(*host)
        run.step(1)
        chhs.lib().chhs_get_state(run.handle, *[chhs._buf(h_, ncell, True)[0] for h_ in host], 0)
    torch.cuda.synchronize()
    e2e_s = reduce_max(time.perf_counter() - t0, world)
    e2e = {"value": units / e2e_s, "unit": UNIT, "h2d_bytes_per_step": 4 * 8 * ncell,
           "d2h_bytes_per_step": 4 * 8 * ncell}

    # roofline of the dominant kernel: the same steps launched kernel by
    # kernel with CUDA events on the solver's stream
    prof = None
    for _ in range(5):
        prof = run.profile_step(prof)
    total_ms = sum(v[0] for v in prof.values())
    dom = max(prof, key=lambda k: prof[k][0])
    sm_ms, sm_launch, sm_units = prof["smooth_finest"]
    flops_per_launch = sm_units / sm_launch * SMOOTH_FLOPS[2]
    # the dominant kernel's duration: finest-level passes back to back between
    # two events on the solver's stream (no per-launch event gaps)
    avg_s = run.profile_smooth(200) / 1e3
    achieved = flops_per_launch / avg_s / 1e12
    traffic = measured_traffic()
    fp64_peak = max(chhs.probe_fp64() for _ in range(3))
    l2_gbs = l2_peak()
    cells_per_launch = sm_units / sm_launch
    hbm_bytes = SMOOTH_BYTES_F64 * cells_per_launch
    hbm_gbs, hbm_src = hbm_peak()
    roofline = {"bound": "alu", "kernel": "k_smooth<double,2,false> on the 512x512 level (FP64 red-black cell update)",
                "achieved": achieved, "peak": fp64_peak, "unit": "TFLOP/s",
                "frac": achieved / fp64_peak,
                "peak_source": "measured: chhs_probe_fp64 (FP64 FMA chains on every SM, best of 3) in this run",
                "peak_nominal": FP64_PEAK_TFLOPS, "frac_of_nominal": achieved / FP64_PEAK_TFLOPS,
                "hbm": {"algorithmic_bytes_per_launch": hbm_bytes, "achieved_gbs": hbm_bytes / avg_s / 1e9,
                        "peak_gbs": hbm_gbs, "peak_source": hbm_src, "frac": hbm_bytes / avg_s / 1e9 / hbm_gbs,
                        "note": "72 B per cell updated (read phi, mu, p, phi^m, phi*, f_mu; write phi, mu, p), "
                                "the hot-path table's byte model; this kernel is bound by the FP64 pipe"},
                "l2": l2_roofline(hbm_bytes, avg_s, l2_gbs, measured_traffic(key="l2_request_bytes_per_launch"),
                                  "the 512^2 hierarchy (~55 MB) stays in the L2 between passes"),
                "traffic": traffic, "flop_per_launch": flops_per_launch,
                "avg_launch_us": 1e6 * avg_s, "avg_launch_us_eager": 1e3 * sm_ms / sm_launch,
                "duration_source": "200 finest-level passes back to back between CUDA events (chhs_profile_smooth)",
                "kernel_shares": {k: round(v[0] / total_ms, 4) for k, v in prof.items()},
                "kernel_us_per_launch": {k: round(1e3 * v[0] / v[1], 2) for k, v in prof.items() if v[1]},
                "largest_share": dom}

    # the mixed-precision form on the same workload and steps, timed the same way
    run32 = chhs.Run(shape, w["h"], w["eps"], w["gamma"], w["dt"], stream=stream.cuda_stream,
                     opts=chhs.default_opts(precision=1))
    run32.set_state(*state0)
    run32.step(args.warmup)
    tuning["mixed"] = run32.autotune(3)
    run32.set_state(*state0)
    barrier(world)
    torch.cuda.synchronize()
    mx_ms, mx_v, mx_resid = time_steps(run32, args.steps, stream, flush)
    mx_max = reduce_max(mx_ms, world)
    run.set_state(*state0)
    run.step(args.steps)
    diff = float(np.max(np.abs(run.get_phi() - run32.get_phi())))
    mprof = None
    run32.set_state(*state0)
    for _ in range(5):
        mprof = run32.profile_step(mprof)
    mtot = sum(v[0] for v in mprof.values())
    mixed = {"value": units / (mx_max / 1e3), "unit": UNIT, "ms_per_step": mx_max / args.steps,
             "kernel_shares": {k: round(v[0] / mtot, 4) for k, v in mprof.items()},
             "kernel_us_per_launch": {k: round(1e3 * v[0] / v[1], 2) for k, v in mprof.items() if v[1]},
             "smooth_finest_avg_launch_us": 1e3 * mprof["smooth_finest"][0] / max(1, mprof["smooth_finest"][1]),
             "vcycles_per_step": mx_v / args.steps, "final_resid": mx_resid,
             "dtype": "f32 V-cycles, f64 residual/update/norms",
             "max_abs_phi_diff_vs_f64_after_K_steps": diff}
    run32.close()

    served = batched = None
    if not args.no_request_loop:
        served = served_leg(mixed["value"] / world)
        batched = batched_leg()
    bubbles = bubbles_leg(stream, flush)

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        rate, nsteps, secs = oracle_rate(w)
        model, ncores = cpu_info()
        cpu = {"value": rate, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": "time steps 2..%d of the same 512x512 workload (%.1f s), single-threaded" % (
                   nsteps + 1, secs), "cpu_model": model, "nproc": ncores}
    run.close()
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": max_ms / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": config(world), "vcycles_per_step": vtot / args.steps, "norms_per_step": checks / args.steps, "final_resid": resid,
                "e2e": e2e, "gpu_launches": launches, "roofline": roofline, "mixed": mixed, "served": served, "batched": batched, "bubbles128": bubbles,
                "tuning": tuning,
                "cpu_baseline": cpu,
                "clocks": clocks}
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def main(argv=None):
    args = parse_args(argv)
    if args.profile_run:
        return profile_run(args)
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
