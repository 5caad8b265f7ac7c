"""The serving workload's stream of runs (experiments.serving_runs) on the
host: seeded and reproducible, inside the configuration's ranges, and Poisson
arrivals whose offered work matches the requested rate."""
import numpy as np

from paper_1611_02967_gb300 import experiments as ex


def test_stream_is_seeded_and_in_range():
    a, ua = ex.serving_runs(12)
    b, ub = ex.serving_runs(12)
    assert np.array_equal(ua, ub)
    for x, y in zip(a, b):
        assert x["shape"] == y["shape"] and x["steps"] == y["steps"] and x["eps"] == y["eps"]
        assert np.array_equal(x["phi0"], y["phi0"])
    for r in a:
        d = len(r["shape"])
        n = r["shape"][0]
        assert all(m == n for m in r["shape"])
        assert (d == 2 and n in (128, 256, 512, 1024, 2048) and r["h"] == 0.025) or \
               (d == 3 and n in (64, 128, 256) and r["h"] == 0.05)
        assert 10 <= r["steps"] <= 500
        assert 0.02 <= r["eps"] <= 0.08 and 0.5 <= r["gamma"] <= 4.0
        assert r["phi0"].shape == r["shape"] and r["cells"] == r["phi0"].size
        assert np.all(np.abs(r["phi0"]) <= 1.0 + 1e-12)
    c, _ = ex.serving_runs(12, seed=6)
    assert any(x["shape"] != y["shape"] or x["steps"] != y["steps"] for x, y in zip(a, c))


def test_shortened_step_range():
    runs, _ = ex.serving_runs(40, steps=(10, 50))
    s = [r["steps"] for r in runs]
    assert min(s) >= 10 and max(s) <= 50 and len(set(s)) > 5


def test_arrivals_offer_the_requested_rate():
    runs, u = ex.serving_runs(12)
    work = np.array([r["cells"] * r["steps"] for r in runs], dtype=float)
    t = ex.serve_arrivals(runs, u, 1e9)
    assert np.all(np.diff(t) > 0) and t[0] > 0
    # gaps are exponential with mean (mean work) / rate: the drawn gaps
    # reproduce it exactly from the uniforms
    gaps = np.diff(np.concatenate([[0.0], t]))
    assert np.allclose(gaps, -np.log(1.0 - u) * work.mean() / 1e9)
    t2 = ex.serve_arrivals(runs, u, 2e9)
    assert np.allclose(t2, t / 2)
