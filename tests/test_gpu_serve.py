"""The request loop (chhs_server_*): continuous batching of independent runs.

Runs of different dimension, size, parameters, precision and length are
submitted while others are on the GPU; each must finish with exactly the
phi it gets when run alone through chhs_create/chhs_step (the loop only
interleaves independent runs on separate streams, so bit-for-bit), the
device pool must never be over-committed, and a run too large for the pool
must fail cleanly.
"""
import time

import numpy as np
import pytest

from paper_1611_02967_gb300 import chhs, inputs

pytestmark = pytest.mark.gpu

REQS = [  # (shape, h, eps, gamma, dt, nsteps, precision, seed)
    ((64, 64), 0.05, 0.05, 1.0, 0.01, 12, 0, 1),
    ((128, 128), 0.025, 0.04, 2.0, 0.005, 9, 1, 2),
    ((32, 64), 0.1, 0.08, 0.5, 0.01, 15, 0, 3),
    ((16, 16, 16), 0.1, 0.08, 2.0, 0.005, 6, 0, 4),
    ((96, 96), 0.05, 0.06, 4.0, 0.005, 7, 1, 5),
    ((256, 256), 0.025, 0.05, 1.0, 0.005, 5, 1, 6),
    ((8, 8, 8), 0.2, 0.1, 1.0, 0.01, 10, 1, 7),
    ((24, 40), 0.1, 0.08, 1.0, 0.01, 11, 0, 8),
]


def _alone(shape, h, eps, gamma, dt, nsteps, precision, seed):
    with chhs.Run(shape, h, eps, gamma, dt, opts=chhs.default_opts(precision=precision)) as run:
        run.set_phi(inputs.spinodal(shape, seed, mean=0.0, amplitude=0.4))
        run.step(nsteps)
        return run.get_phi()


def test_each_result_same_alone_and_in_the_mix():
    with chhs.Server(pool_bytes=512 << 20, max_active=6, steps_per_slice=3) as sv:
        ids, max_active = [], 0
        for k, (shape, h, eps, gamma, dt, nsteps, prec, seed) in enumerate(REQS):
            ids.append(sv.submit(shape, h, eps, gamma, dt, nsteps,
                                 inputs.spinodal(shape, seed, mean=0.0, amplitude=0.4), precision=prec))
            if k % 3 == 2:  # later arrivals join while earlier runs are on the GPU
                time.sleep(0.002)
            max_active = max(max_active, sv.stats()["active"])
        for rid in ids:
            assert sv.wait(rid, 120.0)
            max_active = max(max_active, sv.stats()["active"])
        results = [sv.result(rid) for rid in ids]
        assert sv.stats()["pool_in_use"] == 0
    assert max_active >= 2  # work overlapped on the device
    for res, req in zip(results, REQS):
        assert res["done"] and res["status"] == chhs.CHHS_OK
        assert res["t_submit"] <= res["t_admit"] <= res["t_done"]
        assert np.array_equal(res["phi"], _alone(*req)), req


def test_admission_by_memory_and_oom():
    shape = (128, 128)
    need = chhs.workspace_bytes(shape)
    with chhs.Server(pool_bytes=2 * need + 4096, max_active=8, steps_per_slice=2) as sv:
        ids = [sv.submit(shape, 0.025, 0.05, 1.0, 0.005, 6, inputs.spinodal(shape, 10 + k, mean=0.0))
               for k in range(5)]
        big = sv.submit((512, 512), 0.025, 0.05, 1.0, 0.005, 2, inputs.spinodal((512, 512), 3, mean=0.0))
        peak = 0
        while any(not sv.result(r, with_phi=False)["done"] for r in ids + [big]):
            st = sv.stats()
            peak = max(peak, st["active"])
            assert st["pool_in_use"] <= 2 * need + 4096
            time.sleep(0.001)
        assert 1 <= peak <= 2  # never more runs than the pool holds
        assert all(sv.result(r)["status"] == chhs.CHHS_OK for r in ids)
        res = sv.result(big)
        assert res["status"] == chhs.CHHS_ERR_OOM
        assert np.isnan(res["phi"]).all()  # refused at admission: it never held a state


def test_serving_stream_through_the_request_loop():
    """The serving workload's generator and driver (the serving study and the
    bench's served leg): a short stream of its runs, submitted as Poisson
    arrivals, all converge and the summary's latencies and throughput are
    consistent with the per-run records."""
    from paper_1611_02967_gb300 import experiments as ex
    runs, u = ex.serving_runs(6, steps=(2, 4))
    res, span = ex.serve(runs, ex.serve_arrivals(runs, u, 2e9))
    assert len(res) == 6 and all(x["status"] == 0 for x in res)
    for x in res:
        assert x["t_submit"] <= x["t_admit"] <= x["t_done"]
    s = ex.serving_summary(runs, res, span, 0.8)
    assert s["all_converged"] and s["runs"] == 6
    assert 0 < s["p50_s"] <= s["p99_s"] <= s["max_s"] <= span + 1e-9
    work = sum(r["cells"] * r["steps"] for r in runs)
    assert abs(s["value"] * span - work) <= 1e-6 * work
