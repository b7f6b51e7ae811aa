"""The seeded synthetic inputs: the named configurations, the batched
instances and the serving trace are reproducible and have the stated shapes."""
import numpy as np

from paper_1312_3004_gb300 import workloads as WL


def test_named_configurations():
    p = WL.params("potts10_L80")
    assert (p["q"], p["L"], p["h"], p["m"]) == (10, 80, 64, 16)
    assert WL.rewl_args(p, 7)[-1] == 7
    paper = WL.params("potts10_L300")
    assert (paper["L"], paper["h"], paper["m"], paper["overlap"]) == (300, 717, 3, 0.75)
    assert WL.params("ising_L8", m=4)["m"] == 4  # overrides


def test_batched_instances_are_reproducible_and_in_range():
    a = WL.batched_instances(2048)
    b = WL.batched_instances(2048)
    assert a == b
    assert len(a) == 2048
    assert {j["q"] for j in a} <= {2, 4, 8, 10}
    assert {j["L"] for j in a} <= set(range(8, 49, 4))
    assert {j["h"] for j in a} <= {4, 8, 16} and {j["m"] for j in a} <= {2, 4}
    assert len({j["seed"] for j in a}) == 2048
    walkers = sum(j["h"] * j["m"] for j in a)
    assert 40000 < walkers < 80000
    assert WL.batched_instances(16, master_seed=1) != WL.batched_instances(16, master_seed=2)


def test_serving_trace_is_a_poisson_stream():
    tr = WL.serving_trace(n=2000)
    assert tr == WL.serving_trace(n=2000)
    t = np.array([x[0] for x in tr])
    assert np.all(np.diff(t) > 0)
    gaps = np.diff(np.concatenate([[0.0], t]))
    assert abs(gaps.mean() - 1 / 50.0) < 0.002  # mean gap 20 ms
    assert abs(gaps.std() / gaps.mean() - 1.0) < 0.1  # exponential: coefficient of variation 1
    for _, j in tr[:200]:
        assert 2 <= j["q"] <= 10 and 6 <= j["L"] <= 12 and 2 <= j["h"] <= 6 and 2 <= j["m"] <= 4


def test_full_serving_trace_has_the_stated_sizes():
    tr = WL.serving_trace_full(n=1000)
    assert tr == WL.serving_trace_full(n=1000)
    t = np.array([x[0] for x in tr])
    gaps = np.diff(np.concatenate([[0.0], t]))
    assert abs(gaps.mean() - 1 / 50.0) < 0.002
    js = [j for _, j in tr]
    assert {j["q"] for j in js} == set(range(2, 11))
    assert min(j["L"] for j in js) >= 16 and max(j["L"] for j in js) <= 96
    assert min(j["h"] for j in js) >= 8 and max(j["h"] for j in js) <= 64
    assert {j["m"] for j in js} == set(range(2, 9))
    assert {j["lnf_final"] for j in js} == {1e-6, 1e-8}
    assert all(j["exchange_interval"] == 10_000 for j in js)


def test_job_cost_estimate_reproduces_its_calibration_runs():
    """The cost model against the converged oracle runs it was fitted to
    (tests/golden/potts10_L{8,12,16,20}_converged.json: median WL steps of
    8 windows x 4 walkers), within a factor 1.3."""
    import json
    import os
    import statistics

    here = os.path.join(os.path.dirname(__file__), "golden")
    for L in (8, 12, 16, 20):
        with open(os.path.join(here, "potts10_L%d_converged.json" % L)) as f:
            runs = json.load(f)["runs"]
        measured = statistics.median(r["wl_steps"] for r in runs)
        est = WL.job_cost_estimate(WL.params("potts10_L%d" % L))
        assert 1 / 1.3 < est / measured < 1.3, (L, est, measured)


def test_weak_scaling_workloads_keep_the_window_width():
    """Sec. 3.1 / Fig. 4: the windows grow in number with N and keep their width;
    at L = 20, 40 and 80 the window formula gives 291 + 1 bins each."""
    from oracle import oracle as O

    for name in ("potts10_L20", "potts10_L40_w291", "potts10_L80_w291"):
        p = WL.params(name)
        assert O.window_table(p["L"], p["h"], p["overlap"])[1] == 291, name
        assert p["m"] == 4 and p["lnf_final"] == 1e-8
